// FP64 pipe peak of the GPU this runs on, for the roofline of the FP64
// propagate kernel (an ALU-bound kernel: its bound is the FP64 pipe, which
// MEASURED_PEAKS-style copy and BF16 GEMM figures do not cover).
//
// Independent FP64 FMA chains (ILP chains per thread) at several launch shapes
// (warps per SM); the best shape is the measured peak.  A second kernel runs
// the same chains in only the first lane of every warp, to show what a warp
// instruction with one active lane costs the pipe.  Prints one JSON line.
// Built and run by bench.py; not part of the library.  With --all it prints
// the detailed table of FP64 / FP32 pipe costs instead (partial-lane warp
// instructions, FP64 MMA against DFMA, the FP64 functions the propagate
// kernel calls in FP64 FMA slots, conversions, FP32 functions).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

template <int ILP>
__global__ void k_dfma(double* out, int iters, double s, int lanes) {
  if ((threadIdx.x & 31) >= lanes) return;
  double a[ILP];
#pragma unroll
  for (int j = 0; j < ILP; j++) a[j] = threadIdx.x * 1e-3 + j;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < ILP; j++) a[j] = fma(a[j], s, 0.999);
  }
  double r = 0;
#pragma unroll
  for (int j = 0; j < ILP; j++) r += a[j];
  if (r == 12345.678) out[0] = r;   // keeps the chains live; never true
}

// FP64 tensor-core MMA (m8n8k4, 512 FLOP per warp instruction) in ILP
// independent accumulator chains; with NF > 0 every MMA is accompanied by NF
// independent DFMAs per lane, to see whether the two share the FP64 pipe.
template <int ILP, int NF>
__global__ void k_dmma(double* out, int iters) {
  const double a = (threadIdx.x & 31) * 1e-3, b = 0.999;
  double c[ILP][2], f[NF > 0 ? NF : 1];
  for (int j = 0; j < ILP; j++) { c[j][0] = j; c[j][1] = j + 0.5; }
  for (int j = 0; j < (NF > 0 ? NF : 1); j++) f[j] = threadIdx.x * 1e-3 + j;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < ILP; j++)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[j][0]), "+d"(c[j][1])
                   : "d"(a), "d"(b));
#pragma unroll
    for (int j = 0; j < NF; j++) f[j] = fma(f[j], 1.0000001, 0.999);
  }
  double r = 0;
  for (int j = 0; j < ILP; j++) r += c[j][0] + c[j][1];
  for (int j = 0; j < NF; j++) r += f[j];
  if (r == 12345.678) out[0] = r;
}

template <int ILP>
__global__ void k_ffma(float* out, int iters, float s) {
  float a[ILP];
  for (int j = 0; j < ILP; j++) a[j] = threadIdx.x * 1e-3f + j;
  for (int i = 0; i < iters; i++)
#pragma unroll
    for (int j = 0; j < ILP; j++) a[j] = fmaf(a[j], s, 0.999f);
  float r = 0;
  for (int j = 0; j < ILP; j++) r += a[j];
  if (r == 12345.678f) out[0] = r;
}

template <int OP>
__global__ void k_dfun(double* out, int iters) {
  double a[4];
  for (int j = 0; j < 4; j++) a[j] = -(threadIdx.x % 7) * 0.1 - 0.5 - 0.01 * j;
  double acc = 0;
  for (int i = 0; i < iters; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      double v;
      if (OP == 0) v = exp(a[j]);
      else if (OP == 1) v = sqrt(-a[j]);
      else if (OP == 2) v = 1.0 / a[j];
      else if (OP == 3) v = erf(a[j]);
      else v = rsqrt(-a[j]);
      acc += v;
      a[j] -= 1e-9;
    }
  if (acc == 12345.678) out[0] = acc;
}

// Conversions and the approximate FP64 reciprocal / reciprocal square root.
__device__ __forceinline__ double rcp_approx_f64(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double rsqrt_approx_f64(double x) {
  double r;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}

template <int OP>
__global__ void k_dmisc(double* out, int iters) {
  double a[4];
  for (int j = 0; j < 4; j++) a[j] = (threadIdx.x % 7) * 0.1 + 0.5 + 0.01 * j;
  double acc = 0;
  for (int i = 0; i < iters; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      double v;
      if (OP == 0) v = (double)((float)a[j] * 1.0001f);          // f64 -> f32 -> f64
      else if (OP == 1) v = rcp_approx_f64(a[j]);
      else if (OP == 2) v = rsqrt_approx_f64(a[j]);
      else v = (double)__double2int_rn(a[j] * 3.0);
      acc += v;
      a[j] += 1e-9;
    }
  if (acc == 12345.678) out[0] = acc;
}

template <int OP>
__global__ void k_ffun(float* out, int iters) {
  float a[4];
  for (int j = 0; j < 4; j++) a[j] = -(threadIdx.x % 7) * 0.1f - 0.5f - 0.01f * j;
  float acc = 0;
  for (int i = 0; i < iters; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      float v;
      if (OP == 0) v = __expf(a[j]);
      else if (OP == 1) v = expf(a[j]);
      else if (OP == 2) v = sqrtf(-a[j]);
      else v = __fdividef(1.f, a[j]);
      acc += v;
      a[j] -= 1e-7f;
    }
  if (acc == 12345.678f) out[0] = acc;
}

template <typename F>
static float best_ms(F launch, int reps) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();
  cudaDeviceSynchronize();
  float best = 1e30f;
  for (int r = 0; r < reps; r++) {
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

static int detailed_table(const cudaDeviceProp& p, double* dout, float* fout) {
  const int sms = p.multiProcessorCount;
  const int blocks = sms * 4, threads = 256;
  const double n8 = (double)blocks * threads * 8, n4 = (double)blocks * threads * 4;
  const int it = 20000, itf = 2000;
  float ms = best_ms([&] { k_dfma<8><<<blocks, threads>>>(dout, it, 1.0000001, 32); }, 5);
  const double dfma = n8 * it / (ms * 1e-3);
  printf("DFMA      %12.4g op/s  %8.3f TFLOP/s\n", dfma, 2 * dfma / 1e12);
  for (int lanes : {1, 8, 16, 24}) {
    const float ml = best_ms([&] { k_dfma<8><<<blocks, threads>>>(dout, it, 1.0000001, lanes); }, 5);
    const double active = (double)blocks * (threads / 32) * lanes * 8 * it;
    printf("DFMA %2d/32 lanes  %10.4g op/s  warp instructions cost %.2fx a full warp's\n", lanes,
           active / (ml * 1e-3), ml / ms);
  }
  {
    // per warp instruction: 8 x 8 x 4 FMA = 256 FMA = 512 FLOP
    const double warps = (double)blocks * threads / 32;
    const float m0 = best_ms([&] { k_dmma<4, 0><<<blocks, threads>>>(dout, it / 4); }, 5);
    const double dmma = warps * 4 * (it / 4) * 256 / (m0 * 1e-3);
    printf("DMMA m8n8k4  %10.4g FMA/s  %8.3f TFLOP/s  (%.2fx DFMA)\n", dmma, 2 * dmma / 1e12, dmma / dfma);
    const float m1 = best_ms([&] { k_dmma<4, 8><<<blocks, threads>>>(dout, it / 4); }, 5);
    const float m2 = best_ms([&] { k_dfma<8><<<blocks, threads>>>(dout, it / 4, 1.0000001, 32); }, 5);
    printf("DMMA x4 + DFMA x8 per iteration: %.3f ms; DMMA alone %.3f ms, DFMA alone %.3f ms (sum %.3f)\n", m1, m0,
           m2, m0 + m2);
  }
  ms = best_ms([&] { k_ffma<8><<<blocks, threads>>>(fout, it, 1.0000001f); }, 5);
  printf("FFMA      %12.4g op/s  %8.3f TFLOP/s  (%.1fx DFMA)\n", n8 * it / (ms * 1e-3), 2 * n8 * it / (ms * 1e-3) / 1e12,
         n8 * it / (ms * 1e-3) / dfma);
  const char* dn[5] = {"exp", "sqrt", "rcp", "erf", "rsqrt"};
  float t[5];
  t[0] = best_ms([&] { k_dfun<0><<<blocks, threads>>>(dout, itf); }, 5);
  t[1] = best_ms([&] { k_dfun<1><<<blocks, threads>>>(dout, itf); }, 5);
  t[2] = best_ms([&] { k_dfun<2><<<blocks, threads>>>(dout, itf); }, 5);
  t[3] = best_ms([&] { k_dfun<3><<<blocks, threads>>>(dout, itf); }, 5);
  t[4] = best_ms([&] { k_dfun<4><<<blocks, threads>>>(dout, itf); }, 5);
  for (int k = 0; k < 5; k++) {
    const double r = n4 * itf / (t[k] * 1e-3);
    printf("%-9s %12.4g op/s  %8.1f FP64 FMA slots\n", dn[k], r, dfma / r);
  }
  const char* mn[4] = {"cvt64-32-64", "rcp.approx.f64", "rsqrt.approx.f64", "d2i_rn+i2d"};
  float tm[4];
  tm[0] = best_ms([&] { k_dmisc<0><<<blocks, threads>>>(dout, itf); }, 5);
  tm[1] = best_ms([&] { k_dmisc<1><<<blocks, threads>>>(dout, itf); }, 5);
  tm[2] = best_ms([&] { k_dmisc<2><<<blocks, threads>>>(dout, itf); }, 5);
  tm[3] = best_ms([&] { k_dmisc<3><<<blocks, threads>>>(dout, itf); }, 5);
  for (int k = 0; k < 4; k++) {
    const double r = n4 * itf / (tm[k] * 1e-3);
    printf("%-17s %12.4g op/s  %8.1f FP64 FMA slots (incl. one DADD)\n", mn[k], r, dfma / r);
  }
  const char* fn[4] = {"__expf", "expf", "sqrtf", "fdividef"};
  float tf[4];
  tf[0] = best_ms([&] { k_ffun<0><<<blocks, threads>>>(fout, it); }, 5);
  tf[1] = best_ms([&] { k_ffun<1><<<blocks, threads>>>(fout, it); }, 5);
  tf[2] = best_ms([&] { k_ffun<2><<<blocks, threads>>>(fout, it); }, 5);
  tf[3] = best_ms([&] { k_ffun<3><<<blocks, threads>>>(fout, it); }, 5);
  for (int k = 0; k < 4; k++) printf("%-9s %12.4g op/s\n", fn[k], n4 * it / (tf[k] * 1e-3));
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int main(int argc, char** argv) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, 0) != cudaSuccess) {
    printf("{\"error\": \"no device\"}\n");
    return 1;
  }
  double* dout = nullptr;
  float* fout = nullptr;
  if (cudaMalloc(&dout, 8) != cudaSuccess || cudaMalloc(&fout, 8) != cudaSuccess) return 1;
  if (argc > 1 && strcmp(argv[1], "--all") == 0) {
    printf("device %s, %d SMs\n", p.name, p.multiProcessorCount);
    return detailed_table(p, dout, fout);
  }
  const int sms = p.multiProcessorCount, threads = 256;
  const int iters = 20000;
  double best = 0.0;
  int best_wps = 0, best_ilp = 0;
  // warps per SM = blocks per SM x 8
  for (int bps : {2, 4, 6, 8}) {
    const int blocks = sms * bps;
    for (int ilp : {8, 16}) {
      const float ms = ilp == 8
                           ? best_ms([&] { k_dfma<8><<<blocks, threads>>>(dout, iters, 1.0000001, 32); }, 5)
                           : best_ms([&] { k_dfma<16><<<blocks, threads>>>(dout, iters / 2, 1.0000001, 32); }, 5);
      const double fma = (double)blocks * threads * 8.0 * iters;   // both shapes do 8 x iters per thread
      const double flops = 2.0 * fma / (ms * 1e-3);
      if (flops > best) { best = flops; best_wps = bps * 8; best_ilp = ilp; }
    }
  }
  // one active lane per warp, same chains: time ratio against all 32 lanes
  const int blocks = sms * (best_wps / 8);
  const float full = best_ms([&] { k_dfma<8><<<blocks, threads>>>(dout, iters, 1.0000001, 32); }, 5);
  const float one = best_ms([&] { k_dfma<8><<<blocks, threads>>>(dout, iters, 1.0000001, 1); }, 5);
  int clk_khz = 0;
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
  const bool ok = cudaGetLastError() == cudaSuccess;
  printf("{\"dfma_gflops\": %.2f, \"warps_per_sm\": %d, \"ilp\": %d, \"one_lane_time_ratio\": %.4f, "
         "\"sms\": %d, \"max_clock_mhz\": %.1f, \"ok\": %s}\n",
         best / 1e9, best_wps, best_ilp, one / full, sms, clk_khz / 1e3, ok ? "true" : "false");
  cudaFree(dout);
  cudaFree(fout);
  return ok ? 0 : 1;
}
