// Single-precision instantiation of the FCH passes (mixed-precision mode).
#define FCH_T float
#define FCH_SUFFIX f32
#include "fch_launch.cuh"
