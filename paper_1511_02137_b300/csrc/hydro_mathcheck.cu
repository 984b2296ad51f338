// Test and measurement support: elementwise evaluation of the device
// arithmetic the sweeps use (hydro_eval_math: reciprocals, recoveries and the
// integer-pipe FP64/FP32 conversions), and the FMA throughput kernels
// that give the roofline its measured ALU peaks (hydro_alu_peak).  Neither has
// a counterpart in the paper; the recovery evaluated here is Eq. 1 with
// p = e/3 inverted in closed form, exactly as the sweeps call it.
#include <cstdint>

#include "hydro.h"
#include "hydro_internal.h"
#include "hydro_math.cuh"

namespace hydro {
namespace {

__global__ void eval_math_kernel(int fn, long long n, const double* __restrict__ in, double* __restrict__ out,
                                 double param) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (fn == HYDRO_MATH_RCP) {
      out[i] = rcp_nr(in[i]);
    } else if (fn == HYDRO_MATH_SQRT_RSQRT) {
      double s, y;
      sqrt_rsqrt_nr(in[i], s, y);
      out[i] = s;
      out[n + i] = y;
    } else if (fn == HYDRO_MATH_D2F) {
      reinterpret_cast<float*>(out)[i] = d2f_rn(in[i]);
    } else if (fn == HYDRO_MATH_F2D) {
      out[i] = f2d(reinterpret_cast<const float*>(in)[i]);
    } else {
      const double E = in[i], Mx = in[n + i], My = in[2 * n + i], Mz = in[3 * n + i];
      int hit = 0;
      double e, vx, vy, vz;
      if (fn == HYDRO_MATH_C2P_FP64) {
        double v2, rden;
        cons_to_prim_rho<MathD>(E, Mx, My, Mz, param, e, vx, vy, vz, v2, rden, hit);
      } else if (fn == HYDRO_MATH_C2P_FP32) {
        // the FP32 path stores the state in FP32 and floors with the rounded e_floor
        float ef, vxf, vyf, vzf, v2f, rdenf;
        cons_to_prim_rho<MathF>((float)E, (float)Mx, (float)My, (float)Mz, (float)param, ef, vxf, vyf, vzf, v2f,
                                rdenf, hit);
        e = ef; vx = vxf; vy = vyf; vz = vzf;
      } else {
        // the mixed path: the FP32 shadow of the FP64 state (E^2 - |M|^2 in FP64), then
        // the recovery the sweeps run from it
        float sh[6], ef, vxf, vyf, vzf, v2f, rdf;
        mixed_shadow(E, Mx, My, Mz, 0.0, param, sh);
        cons_to_prim_shadow_rho(sh[0], sh[1], sh[2], sh[3], sh[5], d2f_rn(param), ef, vxf, vyf, vzf, v2f, rdf, hit);
        e = ef; vx = vxf; vy = vyf; vz = vzf;
      }
      out[i] = e;
      out[n + i] = vx;
      out[2 * n + i] = vy;
      out[3 * n + i] = vz;
      out[4 * n + i] = (double)hit;
    }
  }
}

// Never read by the host: the throughput kernels store their chains' sum here
// only when it takes an impossible value, which keeps the chains alive.
__device__ double g_peak_sink;

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

// kChains independent FMA chains per thread, x <- x a + b, which converge to
// b / (1 - a) and stay normal.
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) alu_peak_kernel(long long iters, float fa, float fb, double da,
                                                                double db) {
  if constexpr (KIND == HYDRO_PEAK_DFMA) {
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * threadIdx.x + k;
#pragma unroll 16
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], da, db);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.0) g_peak_sink = s;
  } else if constexpr (KIND == HYDRO_PEAK_FFMA2) {
    float2 x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = make_float2(1e-3f * threadIdx.x + k, 2e-3f * threadIdx.x + k);
    const float2 a2 = make_float2(fa, fa), b2 = make_float2(fb, fb);
#pragma unroll 16
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k].x + x[k].y;
    if (s == -1.0f) g_peak_sink = s;
  } else {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * threadIdx.x + k;
#pragma unroll 16
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], fa, fb);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.0f) g_peak_sink = s;
  }
}

template <int KIND>
cudaError_t run_peak(long long iters, cudaStream_t s, double* flop, double* ms) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err == cudaSuccess)
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, alu_peak_kernel<KIND>, kPeakThreads, 0);
  if (err != cudaSuccess) return err;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  cudaEvent_t e0, e1;
  err = cudaEventCreate(&e0);
  if (err != cudaSuccess) return err;
  err = cudaEventCreate(&e1);
  if (err != cudaSuccess) {
    cudaEventDestroy(e0);
    return err;
  }
  cudaEventRecord(e0, s);
  alu_peak_kernel<KIND><<<blocks, kPeakThreads, 0, s>>>(iters, 0.999999f, 1e-6f, 0.999999, 1e-6);
  err = cudaGetLastError();
  cudaEventRecord(e1, s);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return err;
  const double lanes = KIND == HYDRO_PEAK_FFMA2 ? 2.0 : 1.0;
  *flop = 2.0 * lanes * kChains * (double)iters * (double)blocks * kPeakThreads;
  *ms = t;
  return cudaSuccess;
}

}  // namespace
}  // namespace hydro

using namespace hydro;

extern "C" hydro_status hydro_eval_math(int32_t fn, int64_t n, const double* d_in, double* d_out, double param,
                                        void* cuda_stream) {
  if (fn < HYDRO_MATH_RCP || fn > HYDRO_MATH_F2D || n < 0 || !d_in || !d_out) return HYDRO_EINVAL;
  if (n == 0) return HYDRO_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const long long blocks = (n + 255) / 256;
  eval_math_kernel<<<(unsigned)(blocks < 148 * 16 ? blocks : 148 * 16), 256, 0, s>>>(fn, n, d_in, d_out, param);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  return err == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

extern "C" hydro_status hydro_alu_peak(int32_t kind, int64_t iters, void* cuda_stream, double* flop, double* ms) {
  if (iters < 1 || !flop || !ms) return HYDRO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t err;
  switch (kind) {
    case HYDRO_PEAK_FFMA: err = run_peak<HYDRO_PEAK_FFMA>(iters, s, flop, ms); break;
    case HYDRO_PEAK_FFMA2: err = run_peak<HYDRO_PEAK_FFMA2>(iters, s, flop, ms); break;
    case HYDRO_PEAK_DFMA: err = run_peak<HYDRO_PEAK_DFMA>(iters, s, flop, ms); break;
    default: return HYDRO_EINVAL;
  }
  return err == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}
