// Shared device helpers: complex arithmetic, bounded grid barrier, P1 stencil coefficients.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hh.h"

namespace hh {

// ---------------------------------------------------------------- complex types
template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <typename T> __host__ __device__ __forceinline__ T mk(double re, double im);
template <> __host__ __device__ __forceinline__ float2 mk<float2>(double re, double im) {
  return make_float2((float)re, (float)im);
}
template <> __host__ __device__ __forceinline__ double2 mk<double2>(double re, double im) {
  return make_double2(re, im);
}
template <typename T> __host__ __device__ __forceinline__ T cadd(T a, T b) { T r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename T> __host__ __device__ __forceinline__ T csub(T a, T b) { T r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename T> __host__ __device__ __forceinline__ T cmul(T a, T b) {
  T r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// acc += a * b
template <typename T> __host__ __device__ __forceinline__ void cfma(T& acc, T a, T b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename T> __host__ __device__ __forceinline__ void cfma_conj(T& acc, T a, T b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
template <typename T, typename S> __host__ __device__ __forceinline__ T cscale(T a, S s) { T r; r.x = a.x * s; r.y = a.y * s; return r; }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ double2 to_d(double2 a) { return a; }

template <typename T> __device__ __forceinline__ T shfl_down(T v, int o) {
  T r; r.x = __shfl_down_sync(0xffffffffu, v.x, o); r.y = __shfl_down_sync(0xffffffffu, v.y, o); return r;
}
template <typename T> __device__ __forceinline__ T shfl_xor(T v, int o) {
  T r; r.x = __shfl_xor_sync(0xffffffffu, v.x, o); r.y = __shfl_xor_sync(0xffffffffu, v.y, o); return r;
}

// ---------------------------------------------------------------- device error word
enum DevErr { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_SINGULAR = 2, DEV_NAN = 3 };

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Words reserved per barrier in a barrier buffer (the counter is the first; the rest keeps
// barriers of different users on separate cache lines).
constexpr int GRID_BAR_WORDS = 64;

// Grid-wide barrier for a cooperative (co-resident) launch.  *count starts at 0 for the
// launch and only grows; `target` is the caller's running arrival target.  Every wait is
// bounded by `budget` SM cycles: on expiry the device error word is set and false is
// returned, so that every CTA leaves the kernel instead of spinning.
__device__ __forceinline__ bool grid_sync(unsigned* count, unsigned& target, int* err, long long budget,
                                          unsigned participants) {
  __shared__ int s_ok;
  __syncthreads();
  target += participants;
  if (threadIdx.x == 0) {
    __threadfence();
    red_release_add(count, 1u);
    long long t0 = clock64();
    int ok = 1;
    while (ld_acquire(count) < target) {
      if (*(volatile int*)err != 0) { ok = 0; break; }
      if (clock64() - t0 > budget) { atomicCAS(err, 0, (int)DEV_TIMEOUT); ok = 0; break; }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}
// the whole grid
__device__ __forceinline__ bool grid_sync(unsigned* count, unsigned& target, int* err, long long budget) {
  return grid_sync(count, target, err, budget, gridDim.x * gridDim.y);
}

// ---------------------------------------------------------------- TMA bulk copies + mbarriers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// one arrival that also announces `bytes` of transaction traffic for the current phase
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// one plain arrival (release at CTA scope)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of an mbarrier.  On expiry the error word is set and the
// wait is retried once more (same budget) so that copies still in flight can land before
// the caller leaves the kernel.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err, long long budget) {
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget) {
      atomicCAS(err, 0, (int)DEV_TIMEOUT);
      const long long t1 = clock64();
      while (!mbar_try_wait(bar, parity) && clock64() - t1 < budget) {
      }
      return false;
    }
  }
  return true;
}
// orders this thread's generic-proxy accesses with its later async-proxy (TMA) accesses
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }
// the same for shared memory only (does not wait for this thread's global loads)
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------- P1 stencil coefficients
// Matrix A = K - k^2 M - i k M_Gamma on the (n+1)^2 grid, cells cut along SW-NE diagonals.
// Right isosceles triangles with legs h: stiffness 1 at the right-angle vertex, 1/2 at the
// two acute ones, -1/2 along a leg, 0 along the hypotenuse; mass h^2/12 (diag), h^2/24 (off);
// boundary edge mass h/3 (diag), h/6 (off).
//
// A node line of type BOT has cells only above it (bottom boundary or a strip's facing
// interface, both impedance), INT cells on both sides, TOP cells only below (impedance).
enum LineType { LINE_BOT = 0, LINE_INT = 1, LINE_TOP = 2 };

struct Coef {
  double k, h;
  int n;
  // The distinct coefficient values, filled once on the host by init(): kernels only select
  // from these tables (GB300's FP64 divide is far too slow to evaluate per thread).
  double2 vert_t[2];      // [edge node i = 0 or n, interior node]
  double diag_t;
  double2 horiz_t[3];     // by line type
  double2 centre_t[3][3]; // [line type][node class: i = 0, interior, i = n]
  // complex64 copies of the vertical and diagonal couplings (the FP64 -> FP32 conversion
  // also runs on the FP64 pipe)
  float2 vert_f[2];
  float diag_f;

  __host__ void init(double k_, int n_) {
    k = k_;
    n = n_;
    h = 1.0 / n_;
    const double kkh = k * k * h * h, kh = k * h;
    // coupling of node (i, l) to (i, l-1): vertical edge shared by up to two triangles,
    // plus the boundary edge mass on the sides x = 0, x = 1
    vert_t[0] = make_double2(1 * (-0.5 - kkh / 24.0), -kh / 6.0);
    vert_t[1] = make_double2(2 * (-0.5 - kkh / 24.0), 0.0);
    // coupling of node (i, l) to (i-1, l-1): the diagonal of one cell (hypotenuse of both halves)
    diag_t = -kkh / 12.0;
    for (int e = 0; e < 2; ++e) vert_f[e] = make_float2((float)vert_t[e].x, (float)vert_t[e].y);
    diag_f = (float)diag_t;
    for (int type = 0; type < 3; ++type) {
      // coupling along a line between (i, l) and (i+1, l)
      const int cnt = (type != LINE_TOP) + (type != LINE_BOT);
      horiz_t[type] = make_double2(cnt * (-0.5 - kkh / 24.0), (type != LINE_INT) ? -kh / 6.0 : 0.0);
      // diagonal entry of node i on a line of the given type
      for (int cls = 0; cls < 3; ++cls) {
        const bool top = type == LINE_TOP, bot = type == LINE_BOT;
        const bool lo_end = cls == 0, hi_end = cls == 2;  // i = 0, i = n
        const bool lt_n = !hi_end, ge_1 = !lo_end;
        int kc = 0, ntri = 0, nbe = 0;
        if (!top && lt_n) { kc += 1; ntri += 2; }  // cell NE of the node: two acute corners
        if (!top && ge_1) { kc += 1; ntri += 1; }  // cell NW: one right-angle corner
        if (!bot && ge_1) { kc += 1; ntri += 2; }  // cell SW: two acute corners
        if (!bot && lt_n) { kc += 1; ntri += 1; }  // cell SE: one right-angle corner
        if (bot || top) nbe += ge_1 + lt_n;
        if (lo_end || hi_end) nbe += (!bot) + (!top);
        centre_t[type][cls] = make_double2(kc - kkh / 12.0 * ntri, -kh / 3.0 * nbe);
      }
    }
  }
  __host__ __device__ double2 vert(int i) const { return vert_t[(i == 0 || i == n) ? 0 : 1]; }
  __host__ __device__ double diag() const { return diag_t; }
  __host__ __device__ double2 horiz(int type) const { return horiz_t[type]; }
  __host__ __device__ double2 centre(int i, int type) const {
    return centre_t[type][i == 0 ? 0 : (i == n ? 2 : 1)];
  }
};

__host__ __device__ __forceinline__ int line_type(int l, int n) {
  return l == 0 ? LINE_BOT : (l == n ? LINE_TOP : LINE_INT);
}

}  // namespace hh
