// aes_batch_regkeys.cu — the batch kernel's 512-thread builds (a span's round
// keys in registers), compiled as a translation unit of their own: the same
// source as aes_batch.cu, whose host entry points launch these through
// launch_batch_regkeys.  Kept apart so that the two builds compile in
// parallel (this file and aes_batch.cu were the longest compiles).
#define AES_BATCH_REGKEYS_TU 1
#include "aes_batch.cu"
