// resample_c2.cu -- kernel instances for one resampling variant.
#include "resample_kernels.cuh"
#define MEGO_VARIANT ::mego::kC2
#include "resample_dispatch.cuh"
