"""GB300-native bulk AES (FIPS-197) in ECB and CTR, after arXiv 1403.7295.

The compute path is hand-written CUDA for sm_103a in ``csrc/``, exposed as the
C ABI of ``include/aesgpu.h`` (``libaesgpu.so``); ``aes`` is its Python
binding.  Importing this package does not load the library; the first call
does, and raises if it has not been built.
"""
from .aes import (  # noqa: F401
    AesError,
    KeySchedule,
    LaunchConfig,
    VARIANT_AUTO,
    VARIANT_BITSLICE,
    VARIANT_TTABLE,
    aes_cbc_decrypt,
    aes_ctr_xcrypt,
    aes_ecb_decrypt,
    aes_ecb_encrypt,
    aes_expand_key,
    aes_xts_decrypt,
    aes_xts_encrypt,
)
