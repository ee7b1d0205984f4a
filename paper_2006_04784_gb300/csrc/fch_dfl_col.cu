// Double-float (FP32 pair) column passes (FCH_FP32X2).
#define FCH_T fch::df
#define FCH_SUFFIX dfl
#define FCH_ONLY_1024
#define FCH_NO_ROW
#include "fch_launch.cuh"
