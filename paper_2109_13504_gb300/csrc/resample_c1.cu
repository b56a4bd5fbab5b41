// resample_c1.cu -- kernel instances for one resampling variant.
#include "resample_kernels.cuh"
#define MEGO_VARIANT ::mego::kC1
#include "resample_dispatch.cuh"
