"""GB300-native learned compressor for sorted integer keys (arXiv 2412.10770).

The compute path is the CUDA library ``liblc.so`` (C ABI in ``include/lc.h``);
``lc`` is its thin Python binding and ``inputs`` the seeded data generators.
"""
from . import inputs  # noqa: F401
from .lc import (Column, LcError, lc_access, lc_access1, lc_compress, lc_compress_batch,  # noqa: F401
                 lc_decode, lc_decode_batch, lc_decode_ranges, lc_deserialize, lc_free, lc_info,
                 lc_lower_bound, lc_lower_bound1, lc_ratio, lc_serialize, lc_size, lc_status, load)
