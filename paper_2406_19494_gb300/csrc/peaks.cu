// FMA-throughput probes: the ALU ceilings the FP64 stencil kernels are compared against.
// Each thread runs 8 independent fused multiply-add chains, so the pipe (not latency) limits.
#include <cuda_runtime.h>

#include "fluid_internal.cuh"

namespace {

template <class T>
__global__ void k_fma_chain(T* out, int iters, T a, T b) {
  T x0 = (T)threadIdx.x, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
    x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
    x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
  }
  const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == (T)-1) out[blockIdx.x] = s;   // never true for these inputs; keeps the chains live
}

template <class T>
int probe(double* gflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FLUID_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FLUID_ECUDA;
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 2048 : 65536;
  T* out = nullptr;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return FLUID_ECUDA;
  k_fma_chain<T><<<blocks, threads, 0, st>>>(out, iters / 8, (T)0.999999, (T)1e-7);   // warm-up
  cudaEventRecord(a, st);
  k_fma_chain<T><<<blocks, threads, 0, st>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(b, st);
  cudaError_t e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess || ms <= 0.f) return FLUID_ECUDA;
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  *gflops = flops / (ms * 1e-3) / 1e9;
  return FLUID_OK;
}

}  // namespace

extern "C" int fluid_measure_peak(int kind, double* gflops, void* stream) {
  if (!gflops || kind < 0 || kind > 1) return FLUID_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return kind == 0 ? probe<double>(gflops, st) : probe<float>(gflops, st);
}

// ---- accuracy check of the kernels' Newton reciprocal against the IEEE division ----------------
#include "flux_math.cuh"

namespace {
__global__ void k_check_rcp(const double* __restrict__ y, double* __restrict__ fast,
                            double* __restrict__ ieee, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    fast[i] = fl::fl_rcp(y[i]);
    ieee[i] = 1.0 / y[i];
  }
}
__global__ void k_check_sqrt(const double* __restrict__ y, double* __restrict__ rs,
                             double* __restrict__ sq, double* __restrict__ ieee, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    rs[i] = fl::fl_rsqrt(y[i]);
    sq[i] = fl::fl_sqrt(y[i]);
    ieee[i] = sqrt(y[i]);
  }
}
}  // namespace

__global__ void k_check_pow(const double* __restrict__ x, double* __restrict__ fast,
                            double* __restrict__ lib, int n, fl::Phys ph) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    fast[i] = fl::viscosity(x[i] * ph.T_ref, ph) / ph.mu_ref;
    lib[i] = exp(ph.visc_exp * log(x[i]));
  }
}

extern "C" int fluid_check_pow(const double* x_dev, double* fast_dev, double* lib_dev, int n,
                               double e, void* stream) {
  if (!x_dev || !fast_dev || !lib_dev || n < 0) return FLUID_EINVAL;
  if (n == 0) return FLUID_OK;
  fl::Phys ph{};
  ph.visc = FLUID_VISC_POWER;
  ph.mu_ref = 1.0;
  ph.T_ref = 1.0;
  ph.iT_ref = 1.0;
  fl::set_power_law(ph, e);
  k_check_pow<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0,
                reinterpret_cast<cudaStream_t>(stream)>>>(x_dev, fast_dev, lib_dev, n, ph);
  return cudaGetLastError() == cudaSuccess ? FLUID_OK : FLUID_ECUDA;
}

extern "C" int fluid_check_sqrt(const double* y_dev, double* rsqrt_dev, double* sqrt_dev,
                                double* ieee_dev, int n, void* stream) {
  if (!y_dev || !rsqrt_dev || !sqrt_dev || !ieee_dev || n < 0) return FLUID_EINVAL;
  if (n == 0) return FLUID_OK;
  k_check_sqrt<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0,
                 reinterpret_cast<cudaStream_t>(stream)>>>(y_dev, rsqrt_dev, sqrt_dev, ieee_dev, n);
  return cudaGetLastError() == cudaSuccess ? FLUID_OK : FLUID_ECUDA;
}

namespace {
__global__ void k_check_widen(const float* __restrict__ x, double* __restrict__ bits,
                              double* __restrict__ cvt, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    bits[i] = fl::fl_widen(x[i]);
    cvt[i] = (double)x[i];
  }
}
}  // namespace

extern "C" int fluid_check_widen(const float* x_dev, double* bits_dev, double* cvt_dev, int n,
                                 void* stream) {
  if (!x_dev || !bits_dev || !cvt_dev || n < 0) return FLUID_EINVAL;
  if (n == 0) return FLUID_OK;
  k_check_widen<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0,
                  reinterpret_cast<cudaStream_t>(stream)>>>(x_dev, bits_dev, cvt_dev, n);
  return cudaGetLastError() == cudaSuccess ? FLUID_OK : FLUID_ECUDA;
}

extern "C" int fluid_check_bulk_staging(const float* src_dev, float* dst_dev, int nrows, int extra_bytes,
                                        unsigned* flags_dev, void* stream) {
  if (!src_dev || !dst_dev || !flags_dev || nrows < 1 || nrows > 8 || extra_bytes < 0 ||
      (reinterpret_cast<uintptr_t>(src_dev) & 15) != 0)
    return FLUID_EINVAL;
  return fl::launch_bulk_probe(src_dev, dst_dev, nrows, (unsigned)extra_bytes, flags_dev,
                               reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? FLUID_OK : FLUID_ECUDA;
}

extern "C" int fluid_check_rcp(const double* y_dev, double* fast_dev, double* ieee_dev, int n,
                               void* stream) {
  if (!y_dev || !fast_dev || !ieee_dev || n < 0) return FLUID_EINVAL;
  if (n == 0) return FLUID_OK;
  k_check_rcp<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0,
                reinterpret_cast<cudaStream_t>(stream)>>>(y_dev, fast_dev, ieee_dev, n);
  return cudaGetLastError() == cudaSuccess ? FLUID_OK : FLUID_ECUDA;
}
