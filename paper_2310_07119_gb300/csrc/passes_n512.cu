// FP32 line passes of length 512.
#define TWA_N 512
#include "passes_inst.inc"
