// Test-only helper: Philox4x32-10 words from cuRAND's device API, for
// comparison with the oracle's own Philox4x32-10 (Salmon et al., SC'11).
//
// cuRAND's Philox state is a 128-bit counter and a 64-bit key: curand_init
// sets key = (lo32(seed), hi32(seed)), adds the subsequence to counter words
// 2-3 and offset / 4 to counter words 0-1, so with an offset that is a
// multiple of four the first curand4() returns Philox4x32-10 of the counter
// (offset / 4 as words 0-1, subsequence as words 2-3) under that key.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

namespace {

__global__ void curand_words(unsigned long long seed, const unsigned long long* sub,
                             const unsigned long long* off, uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed, sub[i], off[i], &st);
  out[i] = curand4(&st);
}

}  // namespace

// Host entry: n counters given as (subsequence, offset) pairs; out receives
// 4 n words.  Returns 0 on success, else the CUDA error code.
extern "C" int curand_philox_words(unsigned long long seed, const unsigned long long* h_sub,
                                   const unsigned long long* h_off, unsigned int* h_out, int n) {
  if (n < 1) return 1;
  unsigned long long* d_sub = nullptr;
  unsigned long long* d_off = nullptr;
  uint4* d_out = nullptr;
  const size_t b8 = sizeof(unsigned long long) * static_cast<size_t>(n);
  const size_t b16 = sizeof(uint4) * static_cast<size_t>(n);
  cudaError_t e = cudaMalloc(&d_sub, b8);
  if (e == cudaSuccess) e = cudaMalloc(&d_off, b8);
  if (e == cudaSuccess) e = cudaMalloc(&d_out, b16);
  if (e == cudaSuccess) e = cudaMemcpy(d_sub, h_sub, b8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_off, h_off, b8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    curand_words<<<(n + 127) / 128, 128>>>(seed, d_sub, d_off, d_out, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h_out, d_out, b16, cudaMemcpyDeviceToHost);
  cudaFree(d_sub);
  cudaFree(d_off);
  cudaFree(d_out);
  return static_cast<int>(e);
}
