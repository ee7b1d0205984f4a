// Double-precision instantiation of the FCH passes.
#define FCH_T double
#define FCH_SUFFIX f64
#include "fch_launch.cuh"
