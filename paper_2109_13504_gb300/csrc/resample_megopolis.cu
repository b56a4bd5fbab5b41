// resample_megopolis.cu -- kernel instances for one resampling variant.
#include "resample_kernels.cuh"
#define MEGO_VARIANT ::mego::kMegopolis
#include "resample_dispatch.cuh"
