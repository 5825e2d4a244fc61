// FP32 line passes of length 256.
#define TWA_N 256
#include "passes_inst.inc"
