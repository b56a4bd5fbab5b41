// resample_metropolis.cu -- kernel instances for one resampling variant.
#include "resample_kernels.cuh"
#define MEGO_VARIANT ::mego::kMetropolis
#include "resample_dispatch.cuh"
