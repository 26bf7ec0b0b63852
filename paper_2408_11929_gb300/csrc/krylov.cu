// Selective flexible multipreconditioned GMRES on the device (Section 3, selection rules of
// Section 4), FP64 complex.  Per iteration, for every active right-hand side r:
//   Z_k = [M_d^{-1} s_d]   (sweep.cu, all directions and right-hand sides in one launch)
//   W   = A Z_k            (matrix-free P1 stencil)
//   block CGS: H = V^H W, W -= V H, twice by default (opts.gs_passes), coefficients summed
//   block QR of W in preconditioner order (the same number of passes against the new vectors),
//     column j deflated when r_jj = 0, or when an earlier column of the block was accepted and
//     r_jj <= eta * ||A z_j|| (the norm of the new column before any Gram-Schmidt)
//   Givens update of the scalar upper Hessenberg matrix, rho = |g_last|, converged when
//     rho / ||b|| <= tol (tested once per iteration)
//   next sources: t = 1 the new vector, t = 2 the other preconditioner's new vector
//     ("cross"), t > 2 the normalised sum of the new vectors ("sum").
// At the end y = R^{-1} g, x = Z y and the explicit residual ||b - A x|| / ||b||.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "common.cuh"
#include "engine.h"
#include "kstate.h"

namespace hh {

void launch_pack(Engine& E, const double2* const* srcptr, const double* scale, int C, int t, int4 codes, void* X);
void launch_unpack(Engine& E, const void* X, int C, int t, int4 codes, double2* dst, size_t stride);
// tensor-core Gram-Schmidt (gs_tc.cu)
cudaError_t gst_set_attributes(int t);
void gst_slice_basis(Engine& E, const KState& K, int S, int mode);
void gst_prepare_columns(Engine& E, const KState& K, int S, const double2* W, bool first);
void gst_inner_products(Engine& E, const KState& K, int S, const double2* W);
void gst_pass_update(Engine& E, const KState& K, int S, double2* W, bool track_max);
int gst_dot_ctas(const Engine& E, const KState& K, int S);
size_t gst_vector_bytes(size_t Dp);
size_t gst_cimage_bytes(int maxV, int t);
int gst_nu_rows(int t);

// ------------------------------------------------------------------ reductions
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* 32 * NV */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int o = 16; o; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[wid * NV + q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0;
      for (int w = 0; w < nw; ++w) s += sh[w * NV + q];
      v[q] = s;
    }
  }
  __syncthreads();
}

// Sum of 32 values over the threads of a block, reduce-scatter style: at each of the five
// warp levels a lane keeps half of its values and receives the partner's half of them, so a
// lane adds 16 + 8 + 4 + 2 + 1 = 31 values instead of 5 x 32 (the adds run on the FP64 pipe,
// the bottleneck of the Gram-Schmidt kernels).  Lane q of the warp ends with value q; the
// warps meet in shared memory and thread q < 32 returns the block's sum of value q.
__device__ __forceinline__ double block_sum32_scatter(double (&v)[32], double* sh /* 32 x warps */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const double send = upper ? v[i] : v[i + h];
      const double keep = upper ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  __syncthreads();
  sh[wid * 32 + lane] = v[0];
  __syncthreads();
  double r = 0;
  if (threadIdx.x < 32)
    for (int w = 0; w < nw; ++w) r += sh[w * 32 + threadIdx.x];
  return r;
}

// ------------------------------------------------------------------ operator
// (A x)(i, j) at node g = j m + i of one column: the P1 stencil of Section 2 (centre, the two
// neighbours on the line, the vertical neighbours and the two diagonal ones).  On interior
// nodes every coefficient is real (the impedance term lives on the boundary), so two FP64
// FMAs per neighbour suffice there instead of four; the dropped products are exact zeros.
__device__ __forceinline__ double2 stencil_row(const double2* __restrict__ xc, size_t g, int i, int j, int n,
                                               const Coef& cf) {
  const int m = n + 1;
  const double dg = cf.diag();
  const int type = line_type(j, n);
  double2 acc;
  if (type == LINE_INT && i >= 1 && i < n) {
    const double c0 = cf.centre_t[LINE_INT][1].x, hz = cf.horiz_t[LINE_INT].x, vt = cf.vert_t[1].x;
    const double2 x0 = xc[g], xe = xc[g + 1], xw = xc[g - 1], xs = xc[g - m], xsw = xc[g - m - 1];
    const double2 xn = xc[g + m], xne = xc[g + m + 1];
    acc.x = c0 * x0.x;             acc.y = c0 * x0.y;
    acc.x = fma(hz, xe.x, acc.x);  acc.y = fma(hz, xe.y, acc.y);
    acc.x = fma(hz, xw.x, acc.x);  acc.y = fma(hz, xw.y, acc.y);
    acc.x = fma(vt, xs.x, acc.x);  acc.y = fma(vt, xs.y, acc.y);
    acc.x = fma(dg, xsw.x, acc.x); acc.y = fma(dg, xsw.y, acc.y);
    acc.x = fma(vt, xn.x, acc.x);  acc.y = fma(vt, xn.y, acc.y);
    acc.x = fma(dg, xne.x, acc.x); acc.y = fma(dg, xne.y, acc.y);
    return acc;
  }
  acc = make_double2(0, 0);
  cfma(acc, cf.centre(i, type), xc[g]);
  const double2 hz = cf.horiz(type);
  if (i + 1 <= n) cfma(acc, hz, xc[g + 1]);
  if (i >= 1) cfma(acc, hz, xc[g - 1]);
  const double2 vt = cf.vert(i);
  if (j >= 1) {
    cfma(acc, vt, xc[g - m]);
    if (i >= 1) { const double2 v = xc[g - m - 1]; acc.x = fma(dg, v.x, acc.x); acc.y = fma(dg, v.y, acc.y); }
  }
  if (j + 1 <= n) {
    cfma(acc, vt, xc[g + m]);
    if (i + 1 <= n) { const double2 v = xc[g + m + 1]; acc.x = fma(dg, v.x, acc.x); acc.y = fma(dg, v.y, acc.y); }
  }
  return acc;
}

// grid (x, ncols): blockIdx.y is the column; 32-bit node indices
__global__ void spmv_kernel(const double2* __restrict__ x, double2* __restrict__ y, int ncols, Coef cf) {
  const int n = cf.n, m = n + 1;
  const unsigned D = (unsigned)m * (unsigned)m;
  const size_t c = blockIdx.y;
  for (unsigned g = blockIdx.x * blockDim.x + threadIdx.x; g < D; g += gridDim.x * blockDim.x) {
    const int j = (int)(g / (unsigned)m), i = (int)(g - (unsigned)j * (unsigned)m);
    y[c * D + g] = stencil_row(x + c * D, g, i, j, n, cf);
  }
}

// y[c] = A x[c] for columns given by pointer tables; grid (x, ncols)
__global__ void spmv_tab_kernel(const double2* const* __restrict__ xcol, double2* const* __restrict__ ycol, int ncols,
                                Coef cf) {
  const int n = cf.n, m = n + 1;
  const unsigned D = (unsigned)m * (unsigned)m;
  const double2* xc = xcol[blockIdx.y];
  double2* yc = ycol[blockIdx.y];
  for (unsigned g = blockIdx.x * blockDim.x + threadIdx.x; g < D; g += gridDim.x * blockDim.x) {
    const int j = (int)(g / (unsigned)m), i = (int)(g - (unsigned)j * (unsigned)m);
    yc[g] = stencil_row(xc, g, i, j, n, cf);
  }
}

// Column tables of one iteration for the active slots act[0..nact): sweep sources, Z
// destinations (= operator inputs) and operator outputs (W).
struct IterTables {
  const double2** src;
  double* scale;
  double2** zdst;
  double2** wdst;
};
__global__ void gather_tables_kernel(KState S, const int* __restrict__ act, int nact, IterTables T,
                                     double2* __restrict__ W) {
  const int t = S.t;
  for (int q = threadIdx.x; q < nact * t; q += blockDim.x) {
    const int a = q / t, d = q % t, r = act[a];
    T.src[q] = S.srcptr[r * t + d];
    T.scale[q] = S.scale[r * t + d];
    T.zdst[q] = S.Zcur[r] + (size_t)d * S.D;
    T.wdst[q] = W + ((size_t)r * t + d) * S.D;
  }
}

// b = -M f_I for Gaussians src rows (x0, y0, sigma, re, im)
__global__ void gauss_nodal_kernel(const double* __restrict__ src, int nsrc, int n, double2* f) {
  const int m = n + 1;
  const double h = 1.0 / n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < (size_t)m * m; g += (size_t)gridDim.x * blockDim.x) {
    const double x = (double)(g % m) * h, yv = (double)(g / m) * h;
    double2 acc = make_double2(0, 0);
    for (int s = 0; s < nsrc; ++s) {
      const double* p = src + 5 * s;
      const double dx = x - p[0], dy = yv - p[1];
      const double e = exp(-(dx * dx + dy * dy) / (2.0 * p[2] * p[2]));
      acc.x += p[3] * e;
      acc.y += p[4] * e;
    }
    f[g] = acc;
  }
}

__global__ void mass_neg_kernel(const double2* __restrict__ f, double2* __restrict__ b, int n) {
  const int m = n + 1;
  const double h = 1.0 / n, h2 = h * h;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < (size_t)m * m; g += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(g / m), i = (int)(g % m);
    const int type = line_type(j, n);
    const bool top = type == LINE_TOP, bot = type == LINE_BOT;
    int ntri = 0;
    if (!top && i < n) ntri += 2;
    if (!top && i >= 1) ntri += 1;
    if (!bot && i >= 1) ntri += 2;
    if (!bot && i < n) ntri += 1;
    double2 acc = cscale(f[g], h2 / 12.0 * ntri);
    const double wh = h2 / 24.0 * ((type != LINE_TOP) + (type != LINE_BOT));
    if (i + 1 <= n) acc = cadd(acc, cscale(f[g + 1], wh));
    if (i >= 1) acc = cadd(acc, cscale(f[g - 1], wh));
    const double wv = h2 / 24.0 * ((i < n) + (i >= 1));
    if (j >= 1) {
      acc = cadd(acc, cscale(f[g - m], wv));
      if (i >= 1) acc = cadd(acc, cscale(f[g - m - 1], h2 / 12.0));
    }
    if (j + 1 <= n) {
      acc = cadd(acc, cscale(f[g + m], wv));
      if (i + 1 <= n) acc = cadd(acc, cscale(f[g + m + 1], h2 / 12.0));
    }
    b[g] = make_double2(-acc.x, -acc.y);
  }
}

// ------------------------------------------------------------------ start / norms
__global__ void norm_part_kernel(const double2* __restrict__ x, size_t D, double* part, int GX, const int* mask) {
  const int r = blockIdx.y;
  if (mask && !mask[r]) return;
  const double2* xr = x + (size_t)r * D;
  double v[1] = {0};
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < D; g += (size_t)GX * blockDim.x) v[0] += cabs2(xr[g]);
  __shared__ double sh[32];
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) part[r * GX + blockIdx.x] = v[0];
}

__global__ void start_kernel(KState S) {
  const int r = blockIdx.x;
  if (threadIdx.x == 0 && S.adm[r]) {
    double s = 0;
    for (int q = 0; q < S.GX; ++q) s += S.npart[r * S.GX + q];
    const double beta = sqrt(s);
    S.beta[r] = beta;
    S.nV[r] = 1;
    S.nZ[r] = 0;
    S.iters[r] = 0;
    S.nacc[r] = 0;
    S.rho[r] = beta;
    S.g[(size_t)r * (S.maxZ + 1)] = make_double2(beta, 0);
    S.Vptr[(size_t)r * S.maxV] = S.V0 + (size_t)r * S.D;
    if (S.gst) {
      S.VSptr[(size_t)r * S.maxV] = S.V0S + (size_t)r * 64 * S.Dp;
      S.vnew0[r] = 0;
      S.vnew1[r] = 1;
    }
    for (int d = 0; d < S.t; ++d) {
      S.srcptr[r * S.t + d] = S.V0 + (size_t)r * S.D;
      S.scale[r * S.t + d] = 1.0;
    }
    if (!(beta > 0)) {
      S.done[r] = 1;
      S.status[r] = (beta == 0) ? HH_OK : HH_ENAN;
    } else {
      S.done[r] = 0;
      S.status[r] = HH_ENOCONV;
    }
  }
}

__global__ void scale_copy_kernel(KState S) {
  const int r = blockIdx.y;
  if (!S.adm[r]) return;
  const double2* b = S.bdev;
  const double beta = S.beta[r];
  const double inv = beta > 0 ? 1.0 / beta : 0.0;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < (size_t)S.D; g += (size_t)gridDim.x * blockDim.x)
    S.V0[(size_t)r * S.D + g] = cscale(b[(size_t)r * S.D + g], inv);
}

// ------------------------------------------------------------------ Gram-Schmidt vs the basis
// The inner products conj(v) w and the updates w - v h run in Gauss's three-multiplication
// form of the complex product (three real FMAs instead of four; the FP64 pipe bounds both
// kernels).  For conj(v) w with dv = Re v - Im v, wd = Im w - Re w, ws = Re w + Im w:
//   a1 = Re w dv,  a2 = Re v wd,  a3 = Im v ws;  Re = a1 + a3,  Im = a1 + a2,
// each of a1, a2, a3 summed over the rows first.  The error stays within a small multiple of
// the unit roundoff times |v| |w| summed over the rows, the normwise bound of the plain form.

// Planes (Re w, Im w - Re w, Re w + Im w) of the new columns, for the first pass's inner products.
template <int TT>
__global__ void __launch_bounds__(256) gs_wprep_kernel(KState S, const double2* __restrict__ W) {
  const int r = blockIdx.y;
  if (S.done[r]) return;
  const size_t D = S.D;
  const double2* Wr = W + (size_t)r * TT * D;
  double* P = S.Wp + (size_t)r * TT * 3 * D;
  __shared__ double sh[32 * TT];
  double n2[TT];
#pragma unroll
  for (int b = 0; b < TT; ++b) n2[b] = 0;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < D; g += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int b = 0; b < TT; ++b) {
      const double2 w = Wr[b * D + g];
      P[(b * 3 + 0) * D + g] = w.x;
      P[(b * 3 + 1) * D + g] = w.y - w.x;
      P[(b * 3 + 2) * D + g] = w.x + w.y;
      n2[b] += cabs2(w);
    }
  }
  // this CTA's part of ||A z_j||^2 (W = A Z before Gram-Schmidt): the deflation reference
  block_sum<TT>(n2, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int b = 0; b < TT; ++b) S.azpart[((size_t)r * TT + b) * gridDim.x + blockIdx.x] = n2[b];
}

template <int TT, int AB>
__global__ void __launch_bounds__(256) gs_dot_kernel(KState S) {
  const int r = blockIdx.y;
  if (S.done[r]) return;
  const int nV = S.nV[r];
  const size_t D = S.D;
  const size_t chunk = (D + S.GX - 1) / S.GX;
  const size_t g0 = blockIdx.x * chunk, g1 = min(D, g0 + chunk);
  const double* P = S.Wp + (size_t)r * TT * 3 * D;
  __shared__ double sh[32 * (AB * TT * 2 > 8 ? AB * TT * 2 : 8)];
  for (int a0 = 0; a0 < nV; a0 += AB) {
    double a1[AB * TT], a2[AB * TT], a3[AB * TT];
#pragma unroll
    for (int q = 0; q < AB * TT; ++q) a1[q] = a2[q] = a3[q] = 0;
    const double2* vp[AB];
#pragma unroll
    for (int ab = 0; ab < AB; ++ab) vp[ab] = (a0 + ab < nV) ? S.Vptr[(size_t)r * S.maxV + a0 + ab] : nullptr;
    // the next row's operands are loaded before this row's multiply-adds (one CTA per SM at
    // this register count: the loads of a row would otherwise stall its warp for a full
    // memory latency)
    double nwr[TT], nwd[TT], nws[TT];
    double2 nvv[AB];
    auto fetch = [&](size_t g) {
#pragma unroll
      for (int b = 0; b < TT; ++b) {
        nwr[b] = P[(b * 3 + 0) * D + g];
        nwd[b] = P[(b * 3 + 1) * D + g];
        nws[b] = P[(b * 3 + 2) * D + g];
      }
#pragma unroll
      for (int ab = 0; ab < AB; ++ab) nvv[ab] = vp[ab] ? vp[ab][g] : make_double2(0, 0);
    };
    if (g0 + threadIdx.x < g1) fetch(g0 + threadIdx.x);
    for (size_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
      double wr[TT], wd[TT], ws[TT];
      double2 vv[AB];
#pragma unroll
      for (int b = 0; b < TT; ++b) { wr[b] = nwr[b]; wd[b] = nwd[b]; ws[b] = nws[b]; }
#pragma unroll
      for (int ab = 0; ab < AB; ++ab) vv[ab] = nvv[ab];
      if (g + blockDim.x < g1) fetch(g + blockDim.x);
#pragma unroll
      for (int ab = 0; ab < AB; ++ab) {
        const double2 v = vv[ab];
        const double dv = v.x - v.y;
#pragma unroll
        for (int b = 0; b < TT; ++b) {
          const int q = ab * TT + b;
          a1[q] = fma(wr[b], dv, a1[q]);
          a2[q] = fma(v.x, wd[b], a2[q]);
          a3[q] = fma(v.y, ws[b], a3[q]);
        }
      }
    }
    double acc[AB * TT * 2];
#pragma unroll
    for (int q = 0; q < AB * TT; ++q) {
      acc[2 * q] = a1[q] + a3[q];
      acc[2 * q + 1] = a1[q] + a2[q];
    }
    if constexpr (AB * TT * 2 == 32) {
      // value q = (ab TT + b) 2 + part lands on thread q
      const double sum = block_sum32_scatter(acc, sh);
      if (threadIdx.x < 32) {
        const int q = threadIdx.x, ab = q / (TT * 2), b = (q / 2) % TT, part = q & 1;
        if (a0 + ab < nV) {
          const size_t p = ((size_t)r * S.maxV + a0 + ab) * TT + b;
          reinterpret_cast<double*>(&S.Hpart[p * S.GX + blockIdx.x])[part] = sum;
        }
      }
    } else {
      block_sum<AB * TT * 2>(acc, sh);
      if (threadIdx.x == 0) {
#pragma unroll
        for (int ab = 0; ab < AB; ++ab) {
          if (a0 + ab < nV) {
#pragma unroll
            for (int b = 0; b < TT; ++b) {
              const size_t p = ((size_t)r * S.maxV + a0 + ab) * TT + b;
              S.Hpart[p * S.GX + blockIdx.x] = make_double2(acc[(ab * TT + b) * 2], acc[(ab * TT + b) * 2 + 1]);
            }
          }
        }
      }
    }
  }
}

// First-pass inner products <v_a, w_b> in FP32 (FP64 data converted on load): with complex64
// sweeps the first Gram-Schmidt pass only has to remove most of w's part in the basis; its
// coefficients c1 (relative error about 1e-6 of |v||w|) are applied by the FP64 update, and the
// FP64 second pass computes the correction c2 of what remains, so that H = c1 + c2, the new
// vectors' orthogonality and the relation A Z = V H stay FP64-accurate.  Same grid and
// partial layout as gs_dot_kernel; per-thread sums of a few terms in FP32, the block sum in FP64.
template <int TT, int AB>
__global__ void __launch_bounds__(256) gs_dot32_kernel(KState S, const double2* __restrict__ W) {
  const int r = blockIdx.y;
  if (S.done[r]) return;
  const int nV = S.nV[r];
  const size_t D = S.D;
  const size_t chunk = (D + S.GX - 1) / S.GX;
  const size_t g0 = blockIdx.x * chunk, g1 = min(D, g0 + chunk);
  const double2* Wr = W + (size_t)r * TT * D;
  __shared__ double sh[32 * (AB * TT * 2 > 8 ? AB * TT * 2 : 8)];
  for (int a0 = 0; a0 < nV; a0 += AB) {
    float ar[AB * TT], ai[AB * TT];
#pragma unroll
    for (int q = 0; q < AB * TT; ++q) ar[q] = ai[q] = 0.f;
    const double2* vp[AB];
#pragma unroll
    for (int ab = 0; ab < AB; ++ab) vp[ab] = (a0 + ab < nV) ? S.Vptr[(size_t)r * S.maxV + a0 + ab] : nullptr;
    for (size_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
      float2 w[TT];
#pragma unroll
      for (int b = 0; b < TT; ++b) {
        const double2 x = Wr[b * D + g];
        w[b] = make_float2((float)x.x, (float)x.y);
      }
#pragma unroll
      for (int ab = 0; ab < AB; ++ab) {
        const double2 vd = vp[ab] ? vp[ab][g] : make_double2(0, 0);
        const float vx = (float)vd.x, vy = (float)vd.y;
#pragma unroll
        for (int b = 0; b < TT; ++b) {
          const int q = ab * TT + b;
          ar[q] = fmaf(vx, w[b].x, fmaf(vy, w[b].y, ar[q]));
          ai[q] = fmaf(vx, w[b].y, fmaf(-vy, w[b].x, ai[q]));
        }
      }
    }
    double acc[AB * TT * 2];
#pragma unroll
    for (int q = 0; q < AB * TT; ++q) {
      acc[2 * q] = ar[q];
      acc[2 * q + 1] = ai[q];
    }
    if constexpr (AB * TT * 2 == 32) {
      const double sum = block_sum32_scatter(acc, sh);
      if (threadIdx.x < 32) {
        const int q = threadIdx.x, ab = q / (TT * 2), b = (q / 2) % TT, part = q & 1;
        if (a0 + ab < nV) {
          const size_t p = ((size_t)r * S.maxV + a0 + ab) * TT + b;
          reinterpret_cast<double*>(&S.Hpart[p * S.GX + blockIdx.x])[part] = sum;
        }
      }
    } else {
      block_sum<AB * TT * 2>(acc, sh);
      if (threadIdx.x == 0) {
#pragma unroll
        for (int ab = 0; ab < AB; ++ab) {
          if (a0 + ab < nV) {
#pragma unroll
            for (int b = 0; b < TT; ++b) {
              const size_t p = ((size_t)r * S.maxV + a0 + ab) * TT + b;
              S.Hpart[p * S.GX + blockIdx.x] = make_double2(acc[(ab * TT + b) * 2], acc[(ab * TT + b) * 2 + 1]);
            }
          }
        }
      }
    }
  }
}

// Grid (pairs / 8, slots), one warp per (basis vector, new column) pair: the lanes take every
// 32nd CTA partial and meet in a fixed shuffle tree (the same order on every run).
__global__ void gs_reduce_kernel(KState S, int first, int gx) {
  const int r = blockIdx.y;
  if (S.done[r]) return;
  const int cnt = S.nV[r] * S.t;
  const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (p >= cnt) return;
  const size_t base = ((size_t)r * S.maxV * S.t + p);
  double2 s = make_double2(0, 0);
  for (int q = lane; q < gx; q += 32) s = cadd(s, S.Hpart[base * S.GX + q]);
#pragma unroll
  for (int o = 16; o; o >>= 1) s = cadd(s, shfl_xor(s, o));
  if (lane == 0) {
    S.Hthis[base] = s;
    S.Hacc[base] = first ? s : cadd(S.Hacc[base], s);
  }
}

// w_b -= sum_a v_a h_ab in the three-multiplication form: with sv = Re v + Im v,
// hd = Im h - Re h, hs = Re h + Im h:  p1 = sum Re h sv, p2 = sum Re v hd, p3 = sum Im v hs,
// Re(v h) summed = p1 - p3, Im = p1 + p2.  write_planes: also store the planes of the updated
// columns for the next pass's inner products.
template <int TT>
__global__ void __launch_bounds__(256) gs_update_kernel(KState S, double2* __restrict__ W, int write_planes) {
  const int r = blockIdx.y;
  if (S.done[r]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nV = S.nV[r];
  double* Hs = reinterpret_cast<double*>(smem_raw);  // nV x TT x (Re h, hd, hs)
  const double2** vps = reinterpret_cast<const double2**>(Hs + (size_t)nV * TT * 3);
  for (int p = threadIdx.x; p < nV * TT; p += blockDim.x) {
    const double2 h = S.Hthis[(size_t)r * S.maxV * TT + p];
    Hs[3 * p] = h.x;
    Hs[3 * p + 1] = h.y - h.x;
    Hs[3 * p + 2] = h.x + h.y;
  }
  for (int a = threadIdx.x; a < nV; a += blockDim.x) vps[a] = S.Vptr[(size_t)r * S.maxV + a];
  __syncthreads();
  const size_t D = S.D;
  double2* Wr = W + (size_t)r * TT * D;
  double* P = S.Wp + (size_t)r * TT * 3 * D;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < D; g += (size_t)gridDim.x * blockDim.x) {
    double p1[TT], p2[TT], p3[TT];
#pragma unroll
    for (int b = 0; b < TT; ++b) p1[b] = p2[b] = p3[b] = 0;
#pragma unroll 4
    for (int a = 0; a < nV; ++a) {
      const double2 v = vps[a][g];
      const double sv = v.x + v.y;
      const double* h = Hs + (size_t)a * TT * 3;
#pragma unroll
      for (int b = 0; b < TT; ++b) {
        p1[b] = fma(h[3 * b], sv, p1[b]);
        p2[b] = fma(v.x, h[3 * b + 1], p2[b]);
        p3[b] = fma(v.y, h[3 * b + 2], p3[b]);
      }
    }
#pragma unroll
    for (int b = 0; b < TT; ++b) {
      double2 w = Wr[b * D + g];
      w.x -= p1[b] - p3[b];
      w.y -= p1[b] + p2[b];
      Wr[b * D + g] = w;
      if (write_planes) {
        P[(b * 3 + 0) * D + g] = w.x;
        P[(b * 3 + 1) * D + g] = w.y - w.x;
        P[(b * 3 + 2) * D + g] = w.x + w.y;
      }
    }
  }
}

// acc -= a b in four FP64 FMAs (the QR kernel is bound by the FP64 pipe; a product followed by a
// subtraction takes six operations)
__device__ __forceinline__ void cfms(double2& acc, double2 a, double2 b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// Sum TT complex values (v[2q], v[2q+1]) over the CTAs of one right-hand side of qr_kernel:
// per-CTA partials into qpart[parity], grid barrier, then every CTA adds the GQ partials with
// all its threads in one fixed order, so that all CTAs hold bit-identical sums (red_out).
template <int TT>
__device__ __forceinline__ bool qr_reduce(double (&v)[2 * TT], const KState& S, int r, int& parity, unsigned* bar,
                                          unsigned& target, int* err, long long budget, double* sh,
                                          double2* red_out) {
  block_sum<2 * TT>(v, sh);
  double2* part = S.qpart + ((size_t)parity * S.nrhs + r) * S.GQ * TT;
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < TT; ++q) part[(size_t)blockIdx.x * TT + q] = make_double2(v[2 * q], v[2 * q + 1]);
  // the CTAs of one right-hand side meet on its own counter: right-hand sides take different
  // numbers of reductions (their deflation decisions differ)
  if (!grid_sync(bar + (size_t)r * GRID_BAR_WORDS, target, err, budget, gridDim.x)) return false;
  double w[2 * TT];
#pragma unroll
  for (int q = 0; q < 2 * TT; ++q) w[q] = 0;
  for (int b = threadIdx.x; b < S.GQ; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < TT; ++q) {
      const double2 p = __ldcg(part + (size_t)b * TT + q);
      w[2 * q] += p.x;
      w[2 * q + 1] += p.y;
    }
  block_sum<2 * TT>(w, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < TT; ++q) red_out[q] = make_double2(w[2 * q], w[2 * q + 1]);
  __syncthreads();
  parity ^= 1;
  return true;
}

// ------------------------------------------------------------------ block QR (cooperative)
// Grid (GQ, nrhs).  Every reduction: per-CTA partials into qpart[parity], a barrier among the
// GQ CTAs of the right-hand side (its own barrier words), then every CTA of the right-hand side
// sums the GQ partials in the same order, so all of them take the same deflation decisions and
// run the same sequence of reductions.
//
// Column j of the block is projected against the accepted vectors q_0..q_{acc-1} (two passes
// by default), its norm r_jj decides deflation, and q_acc = w_j / r_jj.  The phases are fused
// so that each reduction also carries what the next step needs:
//   R1  |w_j|^2 of every column (nu_j, the deflation reference) and <w_0, w_1>;
//   B   (pass 2 only) w_j -= sum c1_q q_q, then the second-pass inner products <q_q, w_j>;
//   C   w_j -= sum c_q q_q (last pass), |w_j|^2, and the first-pass inner products of the next
//       column, <q_q, w_{j+1}> and <w_j, w_{j+1}> (= r_jj <q_acc, w_{j+1}> once w_j is accepted).
// Every thread owns the same elements (g0 + threadIdx.x + k blockDim.x) in every phase, so the
// phases need no synchronisation besides the reductions: t = 4 takes 7 reductions.
template <int TT>
__global__ void __launch_bounds__(256) qr_kernel(KState S, double2* __restrict__ W, unsigned* bar, int* err,
                                                 long long budget) {
  const int r = blockIdx.y;
  const bool active = S.done[r] == 0;
  const size_t D = S.D;
  const size_t chunk = (D + S.GQ - 1) / S.GQ;
  const size_t g0 = blockIdx.x * chunk, g1 = min(D, g0 + chunk);
  double2* Wr = W + (size_t)r * TT * D;
  double2* Vr = S.Vcur[r];
  __shared__ double sh[32 * 8];
  __shared__ double2 red_out[TT];
  const double* ro = reinterpret_cast<const double*>(red_out);
  unsigned target = 0;
  int parity = 0;
  const bool writer = blockIdx.x == 0 && threadIdx.x == 0;
  if (writer && active)
    for (int q = 0; q < TT * TT; ++q) S.Rnew[(size_t)r * TT * TT + q] = make_double2(0, 0);

  auto reduce = [&](double (&v)[2 * TT]) -> bool {
    return qr_reduce<TT>(v, S, r, parity, bar, target, err, budget, sh, red_out);
  };

  // deflation reference ||A z_j||: the GX parts of gs_wprep_kernel, summed in the same order by
  // every CTA (so that all of them take the same decisions)
  double az[TT];
  {
#pragma unroll
    for (int j = 0; j < TT; ++j) az[j] = 0;
    if (active)
      for (int c = threadIdx.x; c < S.GX; c += blockDim.x)
#pragma unroll
        for (int j = 0; j < TT; ++j) az[j] += __ldcg(S.azpart + ((size_t)r * TT + j) * S.GX + c);
    block_sum<TT>(az, sh);
    __shared__ double az_s[TT];
    if (threadIdx.x == 0)
#pragma unroll
      for (int j = 0; j < TT; ++j) az_s[j] = sqrt(az[j]);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < TT; ++j) az[j] = az_s[j];
  }
  // R1: norms in doubles 0..TT-1, <w_0, w_1> in slot NS
  constexpr int NS = (TT + 1) / 2;
  double nu[TT];
  double2 xn = make_double2(0, 0);  // <w_j, w_{j+1}> of the column being decided
  {
    double v[2 * TT];
#pragma unroll
    for (int q = 0; q < 2 * TT; ++q) v[q] = 0;
    if (active)
      for (size_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        double2 wv[TT];
#pragma unroll
        for (int j = 0; j < TT; ++j) {
          wv[j] = Wr[j * D + g];
          v[j] += cabs2(wv[j]);
        }
        if constexpr (TT > 1) {
          double2 x = make_double2(v[2 * NS], v[2 * NS + 1]);
          cfma_conj(x, wv[0], wv[1]);
          v[2 * NS] = x.x;
          v[2 * NS + 1] = x.y;
        }
      }
    if (!reduce(v)) return;
#pragma unroll
    for (int j = 0; j < TT; ++j) nu[j] = sqrt(ro[j]);
    if constexpr (TT > 1) xn = red_out[NS];
  }
  int acc = 0;  // accepted new vectors so far (the same in every CTA)
  int amap[TT];
  double2 dn[TT];  // first-pass coefficients <q_q, w_{j+1}> for the next column
#pragma unroll
  for (int q = 0; q < TT; ++q) dn[q] = make_double2(0, 0);
  double rj = nu[0];  // the first column has nothing to be projected against
#pragma unroll
  for (int j = 0; j < TT; ++j) {
    double2* w = Wr + j * D;
    if (j > 0) {
      double2 cur[TT], tot[TT];
#pragma unroll
      for (int q = 0; q < TT; ++q) cur[q] = tot[q] = dn[q];
      if (acc > 0 && S.passes >= 2) {
        // phase B
        double v[2 * TT];
#pragma unroll
        for (int q = 0; q < 2 * TT; ++q) v[q] = 0;
        if (active)
          for (size_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
            double2 wv = w[g];
#pragma unroll
            for (int q = 0; q < TT - 1; ++q)
              if (q < acc) cfms(wv, cur[q], Vr[q * D + g]);
            w[g] = wv;
#pragma unroll
            for (int q = 0; q < TT - 1; ++q)
              if (q < acc) {
                double2 x = make_double2(v[2 * q], v[2 * q + 1]);
                cfma_conj(x, Vr[q * D + g], wv);
                v[2 * q] = x.x;
                v[2 * q + 1] = x.y;
              }
          }
        if (!reduce(v)) return;
#pragma unroll
        for (int q = 0; q < TT; ++q) {
          cur[q] = q < acc ? red_out[q] : make_double2(0, 0);
          tot[q] = cadd(tot[q], cur[q]);
        }
      }
      // phase C
      const bool next = j + 1 < TT;
      double v[2 * TT];
#pragma unroll
      for (int q = 0; q < 2 * TT; ++q) v[q] = 0;
      if (active)
        for (size_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
          double2 wv = w[g];
          if (acc > 0) {
#pragma unroll
            for (int q = 0; q < TT - 1; ++q)
              if (q < acc) cfms(wv, cur[q], Vr[q * D + g]);
            w[g] = wv;
          }
          v[0] += cabs2(wv);
          if (next) {
            // slot q + 1: <q_q, w_{j+1}> for q < acc, then <w_j, w_{j+1}> (static indices: the
            // slots stay in registers)
            const double2 wn = Wr[(j + 1) * D + g];
#pragma unroll
            for (int q = 0; q < TT - 1; ++q)
              if (q <= acc) {
                double2 x = make_double2(v[2 * (q + 1)], v[2 * (q + 1) + 1]);
                cfma_conj(x, q < acc ? Vr[q * D + g] : wv, wn);
                v[2 * (q + 1)] = x.x;
                v[2 * (q + 1) + 1] = x.y;
              }
          }
        }
      if (!reduce(v)) return;
      rj = sqrt(ro[0]);
#pragma unroll
      for (int q = 0; q < TT; ++q) dn[q] = (next && q < acc) ? red_out[q + 1] : make_double2(0, 0);
      if (next) xn = red_out[acc + 1];
      if (writer && active)
#pragma unroll
        for (int q = 0; q < TT - 1; ++q)
          if (q < acc) {
            double2* p = S.Rnew + (size_t)r * TT * TT + q * TT + j;
            *p = cadd(*p, tot[q]);
          }
    }
    amap[j] = -1;
    // the first accepted column of the block is kept whenever r_jj > 0 (a lucky breakdown when
    // A z lies in the basis' span); later ones must exceed eta ||A z_j||
    if (active && rj > (acc > 0 ? S.eta * az[j] : 0.0) && isfinite(rj)) {
      const double inv = 1.0 / rj;
      double2* vo = Vr + acc * D;
      for (size_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) vo[g] = cscale(w[g], inv);
      if (writer) S.Rnew[(size_t)r * TT * TT + acc * TT + j] = make_double2(rj, 0);
      if (j + 1 < TT)
#pragma unroll
        for (int q = 0; q < TT; ++q)
          if (q == acc) dn[q] = cscale(xn, inv);  // <q_acc, w_{j+1}>, r_jj real
      amap[j] = acc;
      ++acc;
    }
  }
  if (writer && active) {
    S.nacc[r] = acc;
#pragma unroll
    for (int j = 0; j < TT; ++j) {
      S.amap[r * TT + j] = amap[j];
      S.nu[r * TT + j] = nu[j];
    }
  }
}

// ------------------------------------------------------------------ Hessenberg / Givens
__device__ void givens(double2 a, double2 b, double& c, double2& s) {
  const double aa = sqrt(cabs2(a)), bb = sqrt(cabs2(b));
  if (bb == 0) { c = 1; s = make_double2(0, 0); return; }
  if (aa == 0) { c = 0; s = make_double2(b.x / bb, -b.y / bb); return; }
  const double rr = hypot(aa, bb);
  c = aa / rr;
  const double2 ph = make_double2(a.x / aa, a.y / aa);
  s = cmul(ph, make_double2(b.x / rr, -b.y / rr));
}

// One warp per slot.  The new Hessenberg columns, the stored rotations (when they fit, `stage`)
// and the block R are loaded by all lanes into shared memory (one memory latency instead of
// one per element).  The rotations of earlier iterations act on every new column alike, so lane
// j applies them to column j (the columns in parallel); then lane 0 takes the columns in order,
// applying the rotations the block's earlier columns generated and generating the column's own
// (inherently sequential).  Each column sees the same operations in the same order as one lane
// applying all of them.
// mode bit 0: the columns in shared memory (else in S.hcol); bit 1: the rotations staged there too
__global__ void hess_kernel(KState S, int mode) {
  const bool cols_smem = (mode & 1) != 0, stage = (mode & 2) != 0;
  const int r = blockIdx.x, lane = threadIdx.x;
  // the basis vectors this step adds, for the slicing of the tensor-core Gram-Schmidt: none
  // unless the step ends normally below
  if (S.gst && lane == 0) S.vnew1[r] = S.vnew0[r];
  if (S.done[r]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = S.t;
  const int ld = S.maxZ + 2;
  // the t new Hessenberg columns (maxZ + 2 entries each), then the rotations: staged copies, or
  // the stored arrays themselves
  double2* cols = cols_smem ? reinterpret_cast<double2*>(smem_raw) : S.hcol + (size_t)r * t * ld;
  double2* rot = reinterpret_cast<double2*>(smem_raw) + (cols_smem ? (size_t)t * ld : 0);
  double2* snS = stage ? rot : S.sn + (size_t)r * S.maxZ;
  double* csS = stage ? reinterpret_cast<double*>(rot + S.maxZ) : S.cs + (size_t)r * S.maxZ;
  const int nold = S.nV[r], nacc = S.nacc[r];
  const size_t D = S.D;
  double2* g = S.g + (size_t)r * (S.maxZ + 1);
  if (nacc == 0) {
    if (lane == 0) {
      S.status[r] = HH_EBREAKDOWN;
      S.done[r] = 1;
    }
    return;
  }
  int nZ = S.nZ[r];
  const int nZ0 = nZ;
  if (stage)
    for (int i = lane; i < nZ; i += blockDim.x) {
      csS[i] = S.cs[(size_t)r * S.maxZ + i];
      snS[i] = S.sn[(size_t)r * S.maxZ + i];
    }
  for (int j = 0; j < t; ++j) {
    const int pos = S.amap[r * t + j];
    if (pos < 0) continue;
    double2* cj = cols + (size_t)j * ld;
    for (int i = lane; i < nold; i += blockDim.x) cj[i] = S.Hacc[((size_t)r * S.maxV + i) * t + j];
    for (int q = lane; q <= pos; q += blockDim.x) cj[nold + q] = S.Rnew[(size_t)r * t * t + q * t + j];
  }
  __syncwarp();
  // the rotations of earlier iterations, the same for every new column: one lane per column
  if (lane < t && S.amap[r * t + lane] >= 0) {
    double2* cj = cols + (size_t)lane * ld;
    for (int i = 0; i < nZ0; ++i) {
      const double cs = csS[i];
      const double2 sn = snS[i];
      const double2 a0 = cj[i], a1 = cj[i + 1];
      cj[i] = cadd(cscale(a0, cs), cmul(sn, a1));
      const double2 msc = make_double2(-sn.x, sn.y);  // -conj(sn)
      cj[i + 1] = cadd(cmul(msc, a0), cscale(a1, cs));
    }
  }
  __syncwarp();
  for (int j = 0; j < t; ++j) {
    const int pos = S.amap[r * t + j];
    if (pos < 0) continue;
    const int c = nZ;  // == nold + pos - 1: this column's entries 0 .. c + 1
    double2* cj = cols + (size_t)j * ld;
    if (lane == 0) {
      // the rotations this iteration's earlier columns generated, then this column's own
      for (int i = nZ0; i < c; ++i) {
        const double cs = csS[i];
        const double2 sn = snS[i];
        const double2 a0 = cj[i], a1 = cj[i + 1];
        cj[i] = cadd(cscale(a0, cs), cmul(sn, a1));
        const double2 msc = make_double2(-sn.x, sn.y);
        cj[i + 1] = cadd(cmul(msc, a0), cscale(a1, cs));
      }
      double cs;
      double2 sn;
      givens(cj[c], cj[c + 1], cs, sn);
      cj[c] = cadd(cscale(cj[c], cs), cmul(sn, cj[c + 1]));
      csS[c] = cs;
      snS[c] = sn;
      if (stage) {
        S.cs[(size_t)r * S.maxZ + c] = cs;
        S.sn[(size_t)r * S.maxZ + c] = sn;
      }
      const double2 g0 = g[c];
      g[c] = cscale(g0, cs);
      g[c + 1] = cmul(make_double2(-sn.x, sn.y), g0);
      S.Zptr[(size_t)r * S.maxZ + c] = S.Zcur[r] + (size_t)j * D;
    }
    __syncwarp();
    double2* Rc = S.Rrot + (size_t)r * ((size_t)S.maxZ * (S.maxZ + 1) / 2) + (size_t)c * (c + 1) / 2;
    for (int i = lane; i <= c; i += blockDim.x) Rc[i] = cj[i];
    __syncwarp();
    nZ = c + 1;
  }
  for (int q = lane; q < nacc; q += blockDim.x) {
    S.Vptr[(size_t)r * S.maxV + nold + q] = S.Vcur[r] + (size_t)q * D;
    if (S.gst) S.VSptr[(size_t)r * S.maxV + nold + q] = S.VScur[r] + (size_t)q * 64 * S.Dp;
  }
  if (S.gst && lane == 0) {
    S.vnew0[r] = nold;
    S.vnew1[r] = nold + nacc;
  }
  __syncwarp();
  if (lane != 0) return;
  S.nV[r] = nold + nacc;
  S.nZ[r] = nZ;
  const int it = S.iters[r] + 1;
  S.iters[r] = it;
  const double rho = sqrt(cabs2(g[nZ]));
  S.rho[r] = rho;
  S.hist[(size_t)r * S.maxit + it - 1] = rho / S.beta[r];
  if (!isfinite(rho)) { S.status[r] = HH_ENAN; S.done[r] = 1; }
  else if (rho / S.beta[r] <= S.tolv[r]) { S.status[r] = HH_OK; S.done[r] = 1; }
  else if (it >= S.maxit) { S.status[r] = HH_ENOCONV; S.done[r] = 1; }
}

// next sources: sum of the new vectors (t > 2), with its norm
__global__ void source_sum_kernel(KState S) {
  const int r = blockIdx.y;
  if (S.done[r] || S.scheme != HH_SCHEME_SUM) return;
  const int nacc = S.nacc[r];
  const size_t D = S.D;
  const double2* Vr = S.Vcur[r];
  double2* s = S.sbuf + (size_t)r * D;
  double v[1] = {0};
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < D; g += (size_t)S.GX * blockDim.x) {
    double2 a = make_double2(0, 0);
    for (int q = 0; q < nacc; ++q) a = cadd(a, Vr[q * D + g]);
    s[g] = a;
    v[0] += cabs2(a);
  }
  __shared__ double sh[32];
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) S.npart[r * S.GX + blockIdx.x] = v[0];
}

__global__ void source_final_kernel(KState S) {
  const int r = blockIdx.x;
  if (threadIdx.x != 0 || S.done[r]) return;
  const int t = S.t;
  const size_t D = S.D;
  const double2* Vr = S.Vcur[r];
  if (S.scheme == HH_SCHEME_SUM) {
    double s = 0;
    for (int q = 0; q < S.GX; ++q) s += S.npart[r * S.GX + q];
    const double nrm = sqrt(s);
    for (int d = 0; d < t; ++d) {
      S.srcptr[r * t + d] = S.sbuf + (size_t)r * D;
      S.scale[r * t + d] = nrm > 0 ? 1.0 / nrm : 0.0;
    }
  } else {
    // cross (and t = 1): preconditioner d takes the new vector built from column (d+1) mod t,
    // or the first surviving one
    for (int d = 0; d < t; ++d) {
      const int jj = (d + 1) % t;
      const int pos = S.amap[r * t + jj];
      S.srcptr[r * t + d] = Vr + (size_t)(pos >= 0 ? pos : 0) * D;
      S.scale[r * t + d] = 1.0;
    }
  }
}

// ------------------------------------------------------------------ final solution
// y = R^-1 g by columns, one warp per slot: once y_i is known, the lanes subtract R(k, i) y_i
// from the right-hand side of every row k < i (column i of the packed R is contiguous), so
// each column costs one memory latency rather than one per entry.
__global__ void backsub_kernel(KState S) {
  const int r = blockIdx.x, lane = threadIdx.x;
  if (!S.fin[r]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sv = reinterpret_cast<double2*>(smem_raw);  // maxZ: right-hand side being reduced
  const int nZ = S.nZ[r];
  const double2* Rb = S.Rrot + (size_t)r * ((size_t)S.maxZ * (S.maxZ + 1) / 2);
  const double2* g = S.g + (size_t)r * (S.maxZ + 1);
  double2* y = S.y + (size_t)r * S.maxZ;
  for (int k = lane; k < nZ; k += blockDim.x) sv[k] = g[k];
  __syncwarp();
  for (int i = nZ - 1; i >= 0; --i) {
    const double2* Ri = Rb + (size_t)i * (i + 1) / 2;  // column i: R(0..i, i)
    const double2 d = Ri[i];
    const double dd = cabs2(d);
    const double2 yi = cmul(sv[i], make_double2(d.x / dd, -d.y / dd));
    __syncwarp();
    if (lane == 0) y[i] = yi;
    for (int k = lane; k < i; k += blockDim.x) sv[k] = csub(sv[k], cmul(Ri[k], yi));
    __syncwarp();
  }
}

__global__ void xsol_kernel(KState S) {
  const int r = blockIdx.y;
  if (!S.fin[r]) return;
  double2* x = S.xout[r];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nZ = S.nZ[r];
  double2* ys = reinterpret_cast<double2*>(smem_raw);
  const double2** zp = reinterpret_cast<const double2**>(ys + S.maxZ);
  for (int c = threadIdx.x; c < nZ; c += blockDim.x) {
    ys[c] = S.y[(size_t)r * S.maxZ + c];
    zp[c] = S.Zptr[(size_t)r * S.maxZ + c];
  }
  __syncthreads();
  const size_t D = S.D;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < D; g += (size_t)gridDim.x * blockDim.x) {
    double2 a = make_double2(0, 0);
    for (int c = 0; c < nZ; ++c) cfma(a, zp[c][g], ys[c]);
    x[g] = a;
  }
}

__global__ void resid_part_kernel(KState S, const double2* __restrict__ W) {
  const int r = blockIdx.y;
  if (!S.fin[r]) return;
  const size_t D = S.D;
  const int GX = S.GX;
  double* part = S.npart;
  const double2* b = S.bdev + (size_t)r * D;
  const double2* Ax = W + (size_t)r * S.t * D;
  double v[1] = {0};
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < D; g += (size_t)GX * blockDim.x) {
    const double2 d = csub(b[g], Ax[g]);
    v[0] += cabs2(d);
  }
  __shared__ double sh[32];
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) part[r * GX + blockIdx.x] = v[0];
}

__global__ void resid_final_kernel(KState S) {
  const int r = blockIdx.x;
  if (threadIdx.x != 0 || !S.fin[r]) return;
  double s = 0;
  for (int q = 0; q < S.GX; ++q) s += S.npart[r * S.GX + q];
  S.res_exp[r] = S.beta[r] > 0 ? sqrt(s) / S.beta[r] : 0.0;
}

int qr_blocks_per_sm() {
  int a = 0, b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, qr_kernel<4>, 256, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, qr_kernel<1>, 256, 0);
  return std::min(a, b);
}

void launch_unpack_tab(Engine& E, const void* X, int C, int t, int4 codes, double2* const* dstcol);

// ------------------------------------------------------------------ slot solver
// Continuous batching: S slots, each an independent MPGMRES solve (its own basis, Hessenberg
// matrix, tolerance and iteration count).  Every iteration sweeps the columns of the active
// slots only; slots finish independently and new right-hand sides are admitted between
// iterations.  Each slot's per-iteration blocks (t columns of Z and of new basis vectors)
// come from a pool of equally sized device blocks and return to it when the slot finishes.
struct SlotSolver::Impl {
  Engine& E;
  int S = 0, t = 0, maxit = 0;
  size_t D = 0;
  KState K{};
  std::vector<void*> owned;
  double2* W = nullptr;       // S * t * D operator outputs / residual scratch
  unsigned* qbar = nullptr;   // per-slot barrier counters of the block QR
  // captured Arnoldi steps, one per number of active slots
  struct StepGraph {
    int nact;
    cudaGraphExec_t exec;
    int64_t kernels;
  };
  std::vector<StepGraph> step_graphs;
  bool step_graph_broken = false;
  int64_t iter_calls = 0;
  static constexpr int HH_EAGAIN_STEP = -1000;
  double2* xstage = nullptr;  // S * D solutions of slots whose caller buffer is host memory
  int* d_act = nullptr;
  IterTables T{};
  // pinned staging
  int *h_act = nullptr, *h_done = nullptr, *h_iters = nullptr, *h_status = nullptr, *h_mask = nullptr;
  double *h_rho = nullptr, *h_beta = nullptr, *h_res = nullptr, *h_tolv = nullptr;
  double2 **h_zcur = nullptr, **h_vcur = nullptr, **h_xout = nullptr, **h_tab0 = nullptr, **h_tab1 = nullptr;
  std::vector<void*> pinned;
  struct Slot {
    bool busy = false, done = false;
    void* tag = nullptr;
    double2* xdev = nullptr;  // where the device solution goes
    double* xuser = nullptr;  // caller buffer (host) or nullptr
    std::vector<void*> blocks;
    std::vector<void*> sblocks;  // slice images of this slot's basis blocks (tensor-core Gram-Schmidt)
  };
  std::vector<Slot> slots;
  std::vector<void*> pool;
  std::vector<void*> spool;  // slice-image blocks (t basis vectors each)
  unsigned char** h_vscur = nullptr;
  int4 codes{};

  explicit Impl(Engine& e) : E(e) {}
  ~Impl() {
    cudaStreamSynchronize(E.stream);
    for (auto& g : step_graphs) cudaGraphExecDestroy(g.exec);
    for (void* p : owned) E.dfree(p);
    for (void* p : pool) E.dfree(p);
    for (void* p : spool) E.dfree(p);
    for (auto& sl : slots) {
      for (void* p : sl.blocks) E.dfree(p);
      for (void* p : sl.sblocks) E.dfree(p);
    }
    for (void* p : pinned) cudaFreeHost(p);
  }
  template <typename T_> T_* dev(size_t count) {
    void* p = nullptr;
    if (E.dmalloc(&p, std::max<size_t>(count * sizeof(T_), 16))) return nullptr;
    cudaMemsetAsync(p, 0, std::max<size_t>(count * sizeof(T_), 16), E.stream);
    owned.push_back(p);
    return reinterpret_cast<T_*>(p);
  }
  template <typename T_> T_* host(size_t count) {
    void* p = nullptr;
    if (cudaMallocHost(&p, std::max<size_t>(count * sizeof(T_), 16)) != cudaSuccess) return nullptr;
    pinned.push_back(p);
    return reinterpret_cast<T_*>(p);
  }
  void* block() {
    if (!pool.empty()) {
      void* p = pool.back();
      pool.pop_back();
      return p;
    }
    void* p = nullptr;
    if (E.dmalloc(&p, (size_t)t * D * sizeof(double2))) return nullptr;
    return p;
  }

  void* sblock() {
    if (!spool.empty()) {
      void* p = spool.back();
      spool.pop_back();
      return p;
    }
    void* p = nullptr;
    if (E.dmalloc(&p, (size_t)t * gst_vector_bytes(K.Dp))) return nullptr;
    return p;
  }

  int init(int nslots) {
    S = nslots;
    t = E.t;
    maxit = E.opts.maxit;
    D = (size_t)E.m * E.m;
    K.nrhs = S; K.t = t; K.D = (int)D; K.maxit = maxit; K.maxV = 1 + maxit * t; K.maxZ = maxit * t;
    K.eta = E.opts.deflate_eta; K.passes = E.opts.gs_passes;
    K.scheme = E.opts.scheme != HH_SCHEME_AUTO ? E.opts.scheme
                                               : (t == 2 ? HH_SCHEME_CROSS : (t > 2 ? HH_SCHEME_SUM : HH_SCHEME_CROSS));
    K.GX = std::max(1, std::min(E.num_sms * 2 / S + 1, (int)((D + 255) / 256)));
    K.GX = std::min(K.GX, E.num_sms * 2);
    const int cap = E.num_sms * E.coop_per_sm;
    // one CTA per SM per slot: every reduction of the block QR meets at a barrier and sums the
    // partials of all GQ CTAs, so more CTAs cost more than the extra parallelism brings
    K.GQ = std::max(1, std::min(cap / S, E.num_sms));
    if (K.GQ * S > cap) return (set_error("too many slots for one cooperative QR launch"), HH_EINVAL);
    K.beta = dev<double>(S); K.done = dev<int>(S); K.status = dev<int>(S);
    K.nV = dev<int>(S); K.nZ = dev<int>(S); K.iters = dev<int>(S); K.nacc = dev<int>(S);
    K.amap = dev<int>((size_t)S * t); K.rho = dev<double>(S); K.nu = dev<double>((size_t)S * t);
    K.cs = dev<double>((size_t)S * K.maxZ); K.sn = dev<double2>((size_t)S * K.maxZ);
    K.hist = dev<double>((size_t)S * maxit); K.npart = dev<double>((size_t)S * K.GX);
    K.azpart = dev<double>((size_t)S * t * K.GX);
    K.Vptr = dev<double2*>((size_t)S * K.maxV); K.Zptr = dev<double2*>((size_t)S * K.maxZ);
    K.Hacc = dev<double2>((size_t)S * K.maxV * t); K.Hthis = dev<double2>((size_t)S * K.maxV * t);
    K.Hpart = dev<double2>((size_t)S * K.maxV * t * K.GX); K.Rnew = dev<double2>((size_t)S * t * t);
    K.g = dev<double2>((size_t)S * (K.maxZ + 1));
    K.Rrot = dev<double2>((size_t)S * ((size_t)K.maxZ * (K.maxZ + 1) / 2));
    K.y = dev<double2>((size_t)S * K.maxZ); K.qpart = dev<double2>((size_t)2 * S * K.GQ * 4);
    K.hcol = dev<double2>((size_t)S * t * (K.maxZ + 2));
    K.sbuf = dev<double2>((size_t)S * D); K.V0 = dev<double2>((size_t)S * D);
    K.srcptr = (const double2**)dev<double2*>((size_t)S * t); K.scale = dev<double>((size_t)S * t);
    K.res_exp = dev<double>(S);
    K.tolv = dev<double>(S); K.Zcur = dev<double2*>(S); K.Vcur = dev<double2*>(S);
    K.adm = dev<int>(S); K.fin = dev<int>(S); K.xout = dev<double2*>(S); K.bdev = dev<double2>((size_t)S * D);
    W = dev<double2>((size_t)S * t * D);
    K.gst = E.opts.gs_tensor ? 1 : 0;
    K.Dp = (int)((D + 767) / 768 * 768);  // whole 256-node groups and 384-node update tiles
    K.NU = gst_nu_rows(t);
    if (K.gst) {
      if (gst_set_attributes(t) != cudaSuccess) {
        cudaGetLastError();
        return (set_error("tensor-core Gram-Schmidt: kernel attributes refused"), HH_ECUDA);
      }
      K.VSptr = dev<unsigned char*>((size_t)S * K.maxV);
      K.VScur = dev<unsigned char*>(S);
      K.V0S = dev<unsigned char>((size_t)S * gst_vector_bytes(K.Dp));
      K.vexp = dev<int>((size_t)S * K.maxV);
      K.vnew0 = dev<int>(S);
      K.vnew1 = dev<int>(S);
      K.vmaxb = dev<unsigned long long>((size_t)S * t);
      K.wmaxb = dev<unsigned long long>((size_t)S * t);
      K.CB = dev<unsigned char>((size_t)S * gst_cimage_bytes(K.maxV, t));
      K.cexp = dev<int>((size_t)S * t);
      h_vscur = host<unsigned char*>(S);
      if (!K.VSptr || !K.V0S || !K.CB || !K.cexp || !h_vscur) return HH_ENOMEM;
    } else {
      K.Wp = dev<double>((size_t)S * t * 3 * D);
      if (!K.Wp) return HH_ENOMEM;
    }
    qbar = dev<unsigned>((size_t)S * GRID_BAR_WORDS);
    xstage = dev<double2>((size_t)S * D);
    d_act = dev<int>(S);
    T.src = (const double2**)dev<double2*>((size_t)S * t); T.scale = dev<double>((size_t)S * t);
    T.zdst = dev<double2*>((size_t)S * t); T.wdst = dev<double2*>((size_t)S * t);
    if (!W || !xstage || !T.wdst || !K.bdev || !K.Rrot) return HH_ENOMEM;
    h_act = host<int>(S); h_done = host<int>(S); h_iters = host<int>(S); h_status = host<int>(S);
    h_mask = host<int>(S); h_rho = host<double>(S); h_beta = host<double>(S); h_res = host<double>(S);
    h_tolv = host<double>(S);
    h_zcur = host<double2*>(S); h_vcur = host<double2*>(S); h_xout = host<double2*>(S);
    h_tab0 = host<double2*>(S); h_tab1 = host<double2*>(S);
    if (!h_tab1) return (set_error("pinned host allocation failed"), HH_ENOMEM);
    for (int r = 0; r < S; ++r) h_done[r] = 1;
    cudaMemcpyAsync(K.done, h_done, sizeof(int) * S, cudaMemcpyHostToDevice, E.stream);
    slots.assign(S, Slot());
    if (E.fd ? fd_reserve(E, S * t) : E.ensure_sweep_ws(S * t)) return HH_ENOMEM;
    int* cp = &codes.x;
    for (int d = 0; d < 4; ++d) cp[d] = d < t ? E.dir_codes[d] : 0;
    cudaError_t e = cudaStreamSynchronize(E.stream);
    if (e != cudaSuccess) return (E.set_cuda_error(e, "slot solver init"), HH_ECUDA);
    return HH_OK;
  }

  int free_slots() const {
    int c = 0;
    for (auto& sl : slots) c += !sl.busy;
    return c;
  }
  int busy() const { return S - free_slots(); }

  // Admit right-hand sides into free slots; returns the number admitted.  b[q] and x[q] may be
  // host or device pointers (unified addressing): a host x is filled when the slot finishes.
  int admit(int count, const double2* const* b, double2* const* x, const double* tol, void* const* tags,
            int* slot_out) {
    for (int r = 0; r < S; ++r) h_mask[r] = 0;
    int used = 0;
    for (int q = 0; q < count; ++q) {
      int r = -1;
      for (int c = 0; c < S; ++c)
        if (!slots[c].busy) { r = c; break; }
      if (r < 0) break;
      cudaPointerAttributes pa{};
      bool x_dev = cudaPointerGetAttributes(&pa, x[q]) == cudaSuccess &&
                   (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
      cudaGetLastError();
      Slot& sl = slots[r];
      sl.busy = true;
      sl.done = false;
      sl.tag = tags ? tags[q] : nullptr;
      sl.xuser = x_dev ? nullptr : reinterpret_cast<double*>(x[q]);
      sl.xdev = x_dev ? x[q] : xstage + (size_t)r * D;
      cudaMemcpyAsync(K.bdev + (size_t)r * D, b[q], D * sizeof(double2), cudaMemcpyDefault, E.stream);
      h_tolv[r] = tol[q];
      h_mask[r] = 1;
      h_xout[r] = sl.xdev;
      if (slot_out) slot_out[q] = r;
      ++used;
    }
    if (!used) return 0;
    cudaMemcpyAsync(K.adm, h_mask, sizeof(int) * S, cudaMemcpyHostToDevice, E.stream);
    cudaMemcpyAsync(K.xout, h_xout, sizeof(double2*) * S, cudaMemcpyHostToDevice, E.stream);
    cudaMemcpyAsync(K.tolv, h_tolv, sizeof(double) * S, cudaMemcpyHostToDevice, E.stream);
    dim3 ng(K.GX, S);
    norm_part_kernel<<<ng, 256, 0, E.stream>>>(K.bdev, D, K.npart, K.GX, K.adm);
    start_kernel<<<S, 32, 0, E.stream>>>(K);
    scale_copy_kernel<<<ng, 256, 0, E.stream>>>(K);
    E.count_launch(3);
    if (K.gst) gst_slice_basis(E, K, S, 1);
    // slots whose right-hand side is zero (or not finite) finish at once
    cudaMemcpyAsync(h_done, K.done, sizeof(int) * S, cudaMemcpyDeviceToHost, E.stream);
    cudaError_t e = cudaStreamSynchronize(E.stream);
    if (e != cudaSuccess) return -(E.set_cuda_error(e, "admit"), HH_ECUDA);
    cudaMemsetAsync(K.adm, 0, sizeof(int) * S, E.stream);
    return used;
  }

  template <int TT>
  // nv: basis vectors of all active slots (each projected against its t new columns)
  void gs_and_qr(cudaError_t& ce, double nv, bool tick) {
    dim3 gsgrid(K.GX, S);
    if (K.gst) {
      for (int pass = 0; pass < K.passes; ++pass) {
        gst_prepare_columns(E, K, S, W, pass == 0);
        if (tick) E.tick_begin(Engine::K_GSDOT);
        gst_inner_products(E, K, S, W);
        // algorithmic: the basis slice images (32 bytes per node and vector) and the new columns
        // (16 t bytes per node, sliced inside the kernel), each read once; one complex
        // multiply-add per basis element and new column
        if (tick) E.tick_end(Engine::K_GSDOT, nv * (double)K.Dp * 32.0 + (double)t * D * 16.0, 8.0 * nv * t * D);
        gs_reduce_kernel<<<dim3((K.maxV * t + 7) / 8, S), 256, 0, E.stream>>>(K, pass == 0, gst_dot_ctas(E, K, S));
        E.count_launch();
        gst_pass_update(E, K, S, W, pass + 1 < K.passes);
      }
      cudaMemsetAsync(qbar, 0, sizeof(unsigned) * S * GRID_BAR_WORDS, E.stream);
      void* args[] = {(void*)&K, (void*)&W, (void*)&qbar, (void*)&E.err, (void*)&E.opts.timeout_cycles};
      ce = E.launch_coop((const void*)qr_kernel<TT>, K.GQ, 256, 0, args, S);
      return;
    }
    gs_wprep_kernel<TT><<<gsgrid, 256, 0, E.stream>>>(K, W);
    E.count_launch();
    for (int pass = 0; pass < K.passes; ++pass) {
      if (tick) E.tick_begin(Engine::K_GSDOT);
      if (pass == 0 && K.passes >= 2 && E.precision == HH_PREC_FP32 && E.opts.gs_first_fp32)
        gs_dot32_kernel<TT, 4><<<gsgrid, 256, 0, E.stream>>>(K, W);
      else
        gs_dot_kernel<TT, 4><<<gsgrid, 256, 0, E.stream>>>(K);
      // one complex multiply-add (8 real flops) per basis element and new column; the basis
      // (16 bytes per element) is read once, the column planes (24 bytes) once per 4 vectors
      if (tick) E.tick_end(Engine::K_GSDOT, nv * D * 16.0 + (double)t * D * 24.0 * nv / 4.0, 8.0 * nv * t * D);
      gs_reduce_kernel<<<dim3((K.maxV * t + 7) / 8, S), 256, 0, E.stream>>>(K, pass == 0, K.GX);
      const size_t smem = (size_t)K.maxV * TT * 3 * sizeof(double) + (size_t)K.maxV * sizeof(void*);
      cudaFuncSetAttribute((const void*)gs_update_kernel<TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      gs_update_kernel<TT><<<gsgrid, 256, smem, E.stream>>>(K, W, pass + 1 < K.passes ? 1 : 0);
      E.count_launch(3);
    }
    cudaMemsetAsync(qbar, 0, sizeof(unsigned) * S * GRID_BAR_WORDS, E.stream);
    void* args[] = {(void*)&K, (void*)&W, (void*)&qbar, (void*)&E.err, (void*)&E.opts.timeout_cycles};
    ce = E.launch_coop((const void*)qr_kernel<TT>, K.GQ, 256, 0, args, S);
  }

  struct Done {
    void* tag;
    int slot;
    hh_result res;
  };

  // One MPGMRES iteration for every active slot; completed slots are finalised into out.
  int iterate(std::vector<Done>& out) {
    int nact = 0;
    for (int r = 0; r < S; ++r)
      if (slots[r].busy && !slots[r].done && !h_done[r]) h_act[nact++] = r;
    if (nact > 0) {
      for (int a = 0; a < nact; ++a) {
        const int r = h_act[a];
        void* z = block();
        void* v = block();
        if (!z || !v) return HH_ENOMEM;
        slots[r].blocks.push_back(z);
        slots[r].blocks.push_back(v);
        h_zcur[r] = (double2*)z;
        h_vcur[r] = (double2*)v;
        if (K.gst) {
          void* sv = sblock();
          if (!sv) return HH_ENOMEM;
          slots[r].sblocks.push_back(sv);
          h_vscur[r] = (unsigned char*)sv;
        }
      }
      if (K.gst) cudaMemcpyAsync(K.VScur, h_vscur, sizeof(unsigned char*) * S, cudaMemcpyHostToDevice, E.stream);
      cudaMemcpyAsync(K.Zcur, h_zcur, sizeof(double2*) * S, cudaMemcpyHostToDevice, E.stream);
      cudaMemcpyAsync(K.Vcur, h_vcur, sizeof(double2*) * S, cudaMemcpyHostToDevice, E.stream);
      cudaMemcpyAsync(d_act, h_act, sizeof(int) * nact, cudaMemcpyHostToDevice, E.stream);
      double nv = 0;  // basis vectors of the active slots before this iteration's block
      for (int a = 0; a < nact; ++a) nv += 1.0 + (double)(slots[h_act[a]].blocks.size() / 2 - 1) * t;
      // Every sample_every()-th iteration of a profiled handle runs eagerly with its kernels timed one class
      // at a time; the others replay the captured step for this number of active slots.
      const bool timed = !E.opts.use_graph || step_graph_broken || (E.opts.profile && iter_calls % E.sample_every() == 0);
      ++iter_calls;
      ++E.iterations_total;
      int rc = HH_OK;
      if (!timed) rc = replay_step(nact, nv);
      if (timed || rc == HH_EAGAIN_STEP) {
        cudaError_t ce = cudaSuccess;
        rc = enqueue_step(nact, nv, true, ce);
        if (ce != cudaSuccess) return (E.set_cuda_error(ce, "qr launch"), HH_ECUDA);
      }
      if (rc) return rc;
    }
    cudaMemcpyAsync(h_done, K.done, sizeof(int) * S, cudaMemcpyDeviceToHost, E.stream);
    cudaError_t se = cudaStreamSynchronize(E.stream);
    if (se != cudaSuccess) return (E.set_cuda_error(se, "iteration"), HH_ECUDA);
    int rc = E.check_device_error("iteration");
    if (rc) return rc;
    return finalize(out);
  }

  // The kernels of one iteration for nact active slots (their tables already on the device).
  // timed: eager, with the per-class timing and the sweep as its own graph; otherwise the
  // launches are being captured, so the sweep is launched inline and nothing is timed.
  int enqueue_step(int nact, double nv, bool timed, cudaError_t& ce) {
    const int C = nact * t;
    gather_tables_kernel<<<1, 256, 0, E.stream>>>(K, d_act, nact, T, W);
    E.count_launch();
    if (E.fd) {
      // the paper's five-point scheme: overlapping-strip sweeps and the five-point operator
      if (timed) E.tick_begin(Engine::K_SWEEP);
      const int frc = fd_precondition(E, T.src, T.scale, C, t, codes, T.zdst, E.opts.single_sweep != 0);
      if (timed) E.tick_end(Engine::K_SWEEP, 0, 0);
      if (frc) return frc;
      if (timed) E.tick_begin(Engine::K_SPMV);
      fd_operator(E, (const double2* const*)T.zdst, T.wdst, C);
      if (timed) E.tick_end(Engine::K_SPMV, 2.0 * C * D * 16.0, 0);
    } else {
      launch_pack(E, T.src, T.scale, C, t, codes, E.w_rin);
      if (timed) E.sample_next_sweep = E.opts.profile != 0;
      int rc = timed ? E.run_sweep(E.w_rin, E.w_v, E.w_w, C, E.opts.single_sweep != 0)
                     : E.sweep_inline(E.w_rin, E.w_v, E.w_w, C, E.opts.single_sweep != 0);
      if (rc) return rc;
      launch_unpack_tab(E, E.w_v, C, t, codes, T.zdst);
      if (timed) E.tick_begin(Engine::K_SPMV);
      spmv_tab_kernel<<<dim3(std::max(1u, E.grid_for(D * C) / C), C), 256, 0, E.stream>>>(T.zdst, T.wdst, C, E.coef);
      E.count_launch();
      if (timed) E.tick_end(Engine::K_SPMV, 2.0 * C * D * 16.0, 0);
    }
    if (timed) E.tick_begin(Engine::K_GS);
    const bool tick_dot = timed;
    switch (t) {
      case 1: gs_and_qr<1>(ce, nv, tick_dot); break;
      case 2: gs_and_qr<2>(ce, nv, tick_dot); break;
      case 3: gs_and_qr<3>(ce, nv, tick_dot); break;
      default: gs_and_qr<4>(ce, nv, tick_dot); break;
    }
    // algorithmic bytes per pass: the basis read twice (FP64: 16 bytes per node and vector;
    // tensor-core form: its 32-byte slice image, by the inner products and by the update) and
    // the new columns (FP64: three planes; slices: their 64 t-byte image, W read and written);
    // the block QR about six passes over the new columns
    if (timed)
      E.tick_end(Engine::K_GS,
                 (K.gst ? K.passes * (2.0 * nv * K.Dp * 32 + 64.0 * C * K.Dp + 2.0 * C * D * 16)
                        : K.passes * (2.0 * nv * D * 16 + 3.0 * C * D * 16)) + 6.0 * C * D * 16,
                 K.passes * 16.0 * nv * t * D);
    if (ce != cudaSuccess) return HH_ECUDA;
    // the Hessenberg column, and the rotations too when they fit in shared memory
    const size_t hcol = (size_t)t * (K.maxZ + 2) * sizeof(double2);
    const size_t hrot = (size_t)K.maxZ * (sizeof(double2) + sizeof(double));
    const int cols_smem = hcol <= 160 * 1024;
    const int stage = (cols_smem ? hcol : 0) + hrot <= 200 * 1024;
    const size_t hsmem = (cols_smem ? hcol : 0) + (stage ? hrot : 0);
    cudaFuncSetAttribute((const void*)hess_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem);
    hess_kernel<<<S, 32, hsmem, E.stream>>>(K, cols_smem | (stage << 1));
    source_sum_kernel<<<dim3(K.GX, S), 256, 0, E.stream>>>(K);
    source_final_kernel<<<S, 32, 0, E.stream>>>(K);
    E.count_launch(3);
    if (K.gst) gst_slice_basis(E, K, S, 0);
    return HH_OK;
  }

  // Replays (capturing on first use) the step graph for nact active slots.  Returns
  // HH_EAGAIN_STEP when the step cannot be captured here; the caller then runs it eagerly
  // and no later step tries again.
  int replay_step(int nact, double nv) {
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
    for (const StepGraph& g : step_graphs)
      if (g.nact == nact) {
        exec = g.exec;
        kernels = g.kernels;
      }
    if (!exec) {
      const int C = nact * t;
      int rc = E.fd ? HH_OK : E.ensure_tuned(C);  // tuning runs kernels and synchronises: not in a capture
      if (rc) return rc;
      cudaGraph_t graph = nullptr;
      const int64_t before = E.kernel_launches;
      cudaError_t ce = cudaStreamBeginCapture(E.stream, cudaStreamCaptureModeThreadLocal);
      if (ce == cudaSuccess) {
        cudaError_t kce = cudaSuccess;
        rc = enqueue_step(nact, nv, false, kce);
        ce = cudaStreamEndCapture(E.stream, &graph);
        if (ce == cudaSuccess && (rc != HH_OK || kce != cudaSuccess)) ce = cudaErrorStreamCaptureInvalidated;
      }
      kernels = E.kernel_launches - before;
      E.kernel_launches = before;
      if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        cudaGetLastError();
        step_graph_broken = true;
        E.step_graph_fallback = true;
        return HH_EAGAIN_STEP;
      }
      step_graphs.push_back(StepGraph{nact, exec, kernels});
      ++E.step_graphs_captured;
    }
    cudaError_t ce = cudaGraphLaunch(exec, E.stream);
    if (ce != cudaSuccess) return (E.set_cuda_error(ce, "step graph launch"), HH_ECUDA);
    E.count_launch((int)kernels);
    return HH_OK;
  }

  // Solution, explicit residual and result of every slot that has just finished.
  int finalize(std::vector<Done>& out) {
    int nfin = 0;
    for (int r = 0; r < S; ++r) {
      h_mask[r] = (slots[r].busy && !slots[r].done && h_done[r]) ? 1 : 0;
      if (h_mask[r]) {
        h_tab0[nfin] = slots[r].xdev;
        h_tab1[nfin] = W + (size_t)r * t * D;
        ++nfin;
      }
    }
    if (!nfin) return HH_OK;
    cudaMemcpyAsync(K.fin, h_mask, sizeof(int) * S, cudaMemcpyHostToDevice, E.stream);
    cudaMemcpyAsync(T.zdst, h_tab0, sizeof(double2*) * nfin, cudaMemcpyHostToDevice, E.stream);
    cudaMemcpyAsync(T.wdst, h_tab1, sizeof(double2*) * nfin, cudaMemcpyHostToDevice, E.stream);
    cudaFuncSetAttribute((const void*)backsub_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(K.maxZ * sizeof(double2)));
    backsub_kernel<<<S, 32, (size_t)K.maxZ * sizeof(double2), E.stream>>>(K);
    const size_t xsmem = (size_t)K.maxZ * (sizeof(double2) + sizeof(void*));
    cudaFuncSetAttribute((const void*)xsol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsmem);
    xsol_kernel<<<dim3(K.GX, S), 256, xsmem, E.stream>>>(K);
    E.tick_begin(Engine::K_SPMV);
    if (E.fd)
      fd_operator(E, (const double2* const*)T.zdst, T.wdst, nfin);
    else
      spmv_tab_kernel<<<dim3(std::max(1u, E.grid_for(D * nfin) / nfin), nfin), 256, 0, E.stream>>>(
          (const double2* const*)T.zdst, T.wdst, nfin, E.coef);
    E.tick_end(Engine::K_SPMV, 2.0 * nfin * D * 16.0, 0);
    resid_part_kernel<<<dim3(K.GX, S), 256, 0, E.stream>>>(K, W);
    resid_final_kernel<<<S, 32, 0, E.stream>>>(K);
    E.count_launch(5);
    cudaMemcpyAsync(h_status, K.status, sizeof(int) * S, cudaMemcpyDeviceToHost, E.stream);
    cudaMemcpyAsync(h_iters, K.iters, sizeof(int) * S, cudaMemcpyDeviceToHost, E.stream);
    cudaMemcpyAsync(h_rho, K.rho, sizeof(double) * S, cudaMemcpyDeviceToHost, E.stream);
    cudaMemcpyAsync(h_beta, K.beta, sizeof(double) * S, cudaMemcpyDeviceToHost, E.stream);
    cudaMemcpyAsync(h_res, K.res_exp, sizeof(double) * S, cudaMemcpyDeviceToHost, E.stream);
    for (int r = 0; r < S; ++r)
      if (h_mask[r] && slots[r].xuser)
        cudaMemcpyAsync(slots[r].xuser, slots[r].xdev, D * sizeof(double2), cudaMemcpyDeviceToHost, E.stream);
    cudaMemsetAsync(K.fin, 0, sizeof(int) * S, E.stream);
    cudaError_t e = cudaStreamSynchronize(E.stream);
    if (e != cudaSuccess) return (E.set_cuda_error(e, "finalize"), HH_ECUDA);
    for (int r = 0; r < S; ++r) {
      if (!h_mask[r]) continue;
      Done d;
      d.tag = slots[r].tag;
      d.slot = r;
      std::memset(&d.res, 0, sizeof(d.res));
      d.res.iterations = h_iters[r];
      d.res.rel_res_implicit = h_beta[r] > 0 ? h_rho[r] / h_beta[r] : 0.0;
      d.res.rel_res_explicit = h_res[r];
      d.res.status = (hh_status)h_status[r];
      out.push_back(d);
      for (void* p : slots[r].blocks) pool.push_back(p);
      slots[r].blocks.clear();
      for (void* p : slots[r].sblocks) spool.push_back(p);
      slots[r].sblocks.clear();
      slots[r] = Slot();
    }
    return HH_OK;
  }
};

SlotSolver::SlotSolver(Engine& E) : impl(new Impl(E)) {}
SlotSolver::~SlotSolver() { delete impl; }
int SlotSolver::init(int slots) { return impl->init(slots); }
int SlotSolver::free_slots() const { return impl->free_slots(); }
int SlotSolver::busy() const { return impl->busy(); }
int SlotSolver::admit(int count, const double2* const* b, double2* const* x, const double* tol, void* const* tags,
                      int* slot_out) {
  return impl->admit(count, b, x, tol, tags, slot_out);
}
int SlotSolver::iterate(std::vector<SlotDone>& out) {
  std::vector<Impl::Done> d;
  const int rc = impl->iterate(d);
  for (auto& q : d) out.push_back(SlotDone{q.tag, q.slot, q.res});
  return rc;
}

int Engine::solve_batch_dev(int nrhs, const double2* b, double2* x, double tol, hh_result* res) {
  if (!batch_solver || batch_slots != nrhs) {
    delete batch_solver;
    batch_solver = nullptr;
    batch_slots = 0;
    auto* fresh = new SlotSolver(*this);
    const int irc = fresh->init(nrhs);
    if (irc) {
      delete fresh;
      return irc;
    }
    batch_solver = fresh;
    batch_slots = nrhs;
  }
  SlotSolver& ss = *batch_solver;
  int rc = HH_OK;
  const size_t D = (size_t)m * m;
  std::vector<const double2*> bp(nrhs);
  std::vector<double2*> xp(nrhs);
  std::vector<double> tv(nrhs, tol);
  std::vector<void*> tags(nrhs);
  for (int r = 0; r < nrhs; ++r) {
    bp[r] = b + (size_t)r * D;
    xp[r] = x + (size_t)r * D;
    tags[r] = reinterpret_cast<void*>((intptr_t)r);
  }
  const int used = ss.admit(nrhs, bp.data(), xp.data(), tv.data(), tags.data(), nullptr);
  if (used < 0) return -used;
  std::vector<SlotDone> done;
  // slots finished at admission (zero right-hand side)
  rc = ss.iterate(done);
  while (rc == HH_OK && ss.busy() > 0) rc = ss.iterate(done);
  collect_ticks();
  if (rc) return rc;
  int worst = HH_OK;
  for (auto& d : done) {
    const int r = (int)(intptr_t)d.tag;
    if (res) res[r] = d.res;
    if (d.res.status != HH_OK && worst == HH_OK) worst = d.res.status;
  }
  return worst;
}

// device tables of column pointers base + c D (the five-point kernels take tables), freed by
// the caller
static int column_table(Engine& E, const double2* base, int ncols, const double2*** out) {
  const size_t D = (size_t)E.m * E.m;
  std::vector<const double2*> hp(ncols);
  for (int c = 0; c < ncols; ++c) hp[c] = base + (size_t)c * D;
  if (E.dmalloc((void**)out, sizeof(void*) * ncols)) return HH_ENOMEM;
  cudaMemcpyAsync(*out, hp.data(), sizeof(void*) * ncols, cudaMemcpyHostToDevice, E.stream);
  return HH_OK;
}

int Engine::apply_operator(int ncols, const double2* x, double2* y) {
  const size_t D = (size_t)m * m;
  tick_begin(K_SPMV);
  if (fd) {
    const double2 **xt = nullptr, **yt = nullptr;
    if (column_table(*this, x, ncols, &xt) || column_table(*this, y, ncols, &yt)) {
      dfree(xt);
      return HH_ENOMEM;
    }
    fd_operator(*this, xt, (double2* const*)yt, ncols);
    cudaStreamSynchronize(stream);
    dfree(xt);
    dfree(yt);
  } else {
    spmv_kernel<<<dim3(std::max(1u, grid_for(D * ncols) / ncols), ncols), 256, 0, stream>>>(x, y, ncols, coef);
  }
  count_launch();
  tick_end(K_SPMV, 2.0 * ncols * D * 16.0, 0);
  cudaError_t e = cudaStreamSynchronize(stream);
  collect_ticks();
  if (e != cudaSuccess) { set_cuda_error(e, "apply_operator"); return HH_ECUDA; }
  return HH_OK;
}

int Engine::assemble_rhs(int nsrc, const double* src_host, double2* rhs) {
  const size_t D = (size_t)m * m;
  double* dsrc = nullptr;
  double2* f = nullptr;
  if (dmalloc((void**)&dsrc, sizeof(double) * 5 * std::max(1, nsrc)) || dmalloc((void**)&f, D * sizeof(double2))) {
    dfree(dsrc);
    return HH_ENOMEM;
  }
  if (nsrc > 0) cudaMemcpyAsync(dsrc, src_host, sizeof(double) * 5 * nsrc, cudaMemcpyHostToDevice, stream);
  if (fd) {
    fd_load(*this, dsrc, nsrc, rhs);  // b = s (-h^2 f), the five-point load vector
  } else {
    gauss_nodal_kernel<<<grid_for(D), 256, 0, stream>>>(dsrc, nsrc, n, f);
    mass_neg_kernel<<<grid_for(D), 256, 0, stream>>>(f, rhs, n);
    count_launch(2);
  }
  cudaError_t e = cudaStreamSynchronize(stream);
  dfree(dsrc);
  dfree(f);
  if (e != cudaSuccess) { set_cuda_error(e, "assemble_rhs"); return HH_ECUDA; }
  return HH_OK;
}

int Engine::apply_preconditioner_dev(int dcode, int ncols, const double2* r, double2* z, bool single) {
  const size_t D = (size_t)m * m;
  if (fd) {
    const double2 **rt = nullptr, **zt = nullptr;
    if (column_table(*this, r, ncols, &rt) || column_table(*this, z, ncols, &zt)) {
      dfree(rt);
      return HH_ENOMEM;
    }
    tick_begin(K_SWEEP);
    const int4 codes = make_int4(dcode, dcode, dcode, dcode);
    int rc = fd_precondition(*this, rt, nullptr, ncols, 1, codes, (double2* const*)zt, single);
    tick_end(K_SWEEP, 0, 0);
    cudaError_t e = cudaStreamSynchronize(stream);
    dfree(rt);
    dfree(zt);
    collect_ticks();
    if (rc) return rc;
    if (e != cudaSuccess) { set_cuda_error(e, "apply_preconditioner"); return HH_ECUDA; }
    return check_device_error("five-point sweep");
  }
  if (ensure_sweep_ws(ncols)) return HH_ENOMEM;
  std::vector<const double2*> hp(ncols);
  std::vector<double> hs(ncols, 1.0);
  for (int c = 0; c < ncols; ++c) hp[c] = r + (size_t)c * D;
  const double2** dp = nullptr;
  double* ds = nullptr;
  if (dmalloc((void**)&dp, sizeof(void*) * ncols) || dmalloc((void**)&ds, sizeof(double) * ncols)) {
    dfree(dp);
    return HH_ENOMEM;
  }
  cudaMemcpyAsync(dp, hp.data(), sizeof(void*) * ncols, cudaMemcpyHostToDevice, stream);
  cudaMemcpyAsync(ds, hs.data(), sizeof(double) * ncols, cudaMemcpyHostToDevice, stream);
  int4 codes = make_int4(dcode, dcode, dcode, dcode);
  launch_pack(*this, dp, ds, ncols, 1, codes, w_rin);
  int rc = run_sweep(w_rin, w_v, w_w, ncols, single);
  if (rc == HH_OK) launch_unpack(*this, w_v, ncols, 1, codes, z, D);
  cudaError_t e = cudaStreamSynchronize(stream);
  dfree(dp);
  dfree(ds);
  collect_ticks();
  if (rc) return rc;
  if (e != cudaSuccess) { set_cuda_error(e, "apply_preconditioner"); return HH_ECUDA; }
  return check_device_error("sweep");
}

}  // namespace hh

namespace hh {

// ------------------------------------------------------------------ one Gram-Schmidt pass
// H = V^H W and W <- W - V H for p basis columns and t new columns (device pointers; H to host
// memory, p x t row-major by basis column), with the solver's own kernels: the tensor-core
// slices when opts.gs_tensor, else the FP64-pipe kernels.  A one-slot kernel state with
// temporary buffers (allocated and freed here).
template <int TT>
static int gs_pass_t(Engine& E, KState& K, double2* W, unsigned char* tmp_slices) {
  const int p = K.maxV;
  dim3 gsgrid(K.GX, 1);
  if (K.gst) {
    std::vector<unsigned char*> sp(p);
    for (int a = 0; a < p; ++a) sp[a] = tmp_slices + (size_t)a * gst_vector_bytes(K.Dp);
    cudaMemcpyAsync(K.VSptr, sp.data(), sizeof(unsigned char*) * p, cudaMemcpyHostToDevice, E.stream);
    for (int c = 0; c < p; c += TT) {
      const int range[2] = {c, std::min(p, c + TT)};
      cudaMemcpyAsync(K.vnew0, &range[0], sizeof(int), cudaMemcpyHostToDevice, E.stream);
      cudaMemcpyAsync(K.vnew1, &range[1], sizeof(int), cudaMemcpyHostToDevice, E.stream);
      gst_slice_basis(E, K, 1, 0);
      cudaStreamSynchronize(E.stream);  // range lives on this stack frame
    }
    gst_prepare_columns(E, K, 1, W, true);
    gst_inner_products(E, K, 1, W);
    gs_reduce_kernel<<<dim3((K.maxV * TT + 7) / 8, 1), 256, 0, E.stream>>>(K, 1, gst_dot_ctas(E, K, 1));
    gst_pass_update(E, K, 1, W, false);
  } else {
    gs_wprep_kernel<TT><<<gsgrid, 256, 0, E.stream>>>(K, W);
    gs_dot_kernel<TT, 4><<<gsgrid, 256, 0, E.stream>>>(K);
    gs_reduce_kernel<<<dim3((K.maxV * TT + 7) / 8, 1), 256, 0, E.stream>>>(K, 1, K.GX);
    const size_t smem = (size_t)K.maxV * TT * 3 * sizeof(double) + (size_t)K.maxV * sizeof(void*);
    if (cudaFuncSetAttribute((const void*)gs_update_kernel<TT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return (set_error("Gram-Schmidt pass: too many basis columns for the FP64 update kernel"), HH_EINVAL);
    gs_update_kernel<TT><<<gsgrid, 256, smem, E.stream>>>(K, W, 0);
  }
  return HH_OK;
}

int gram_schmidt_pass(Engine& E, int p, const double2* V, int t, double2* W, double2* H_host) {
  const size_t D = (size_t)E.m * E.m;
  KState K{};
  std::vector<void*> owned;
  auto dev = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (E.dmalloc(&q, std::max<size_t>(bytes, 16))) return nullptr;
    cudaMemsetAsync(q, 0, std::max<size_t>(bytes, 16), E.stream);
    owned.push_back(q);
    return q;
  };
  struct Free {
    Engine& E;
    std::vector<void*>& v;
    ~Free() {
      cudaStreamSynchronize(E.stream);
      for (void* q : v) E.dfree(q);
    }
  } guard{E, owned};
  K.nrhs = 1; K.t = t; K.D = (int)D; K.maxit = 1; K.maxV = p; K.maxZ = 1; K.passes = 1;
  K.GX = std::max(1, std::min(E.num_sms * 2 + 1, (int)((D + 255) / 256)));
  K.GX = std::min(K.GX, E.num_sms * 2);
  K.gst = E.opts.gs_tensor ? 1 : 0;
  K.Dp = (int)((D + 767) / 768 * 768);
  K.NU = gst_nu_rows(t);
  K.done = (int*)dev(sizeof(int));
  K.nV = (int*)dev(sizeof(int));
  K.adm = (int*)dev(sizeof(int));
  K.Vptr = (double2**)dev(sizeof(double2*) * p);
  K.Hpart = (double2*)dev(sizeof(double2) * p * t * K.GX);
  K.Hthis = (double2*)dev(sizeof(double2) * p * t);
  K.Hacc = (double2*)dev(sizeof(double2) * p * t);
  K.azpart = (double*)dev(sizeof(double) * t * K.GX);
  unsigned char* slices = nullptr;
  if (K.gst) {
    if (gst_set_attributes(t) != cudaSuccess) return (E.set_cuda_error(cudaGetLastError(), "attributes"), HH_ECUDA);
    K.VSptr = (unsigned char**)dev(sizeof(unsigned char*) * p);
    K.vexp = (int*)dev(sizeof(int) * p);
    K.vnew0 = (int*)dev(sizeof(int));
    K.vnew1 = (int*)dev(sizeof(int));
    K.vmaxb = (unsigned long long*)dev(sizeof(unsigned long long) * t);
    K.wmaxb = (unsigned long long*)dev(sizeof(unsigned long long) * t);
    K.CB = (unsigned char*)dev(gst_cimage_bytes(p, t));
    K.cexp = (int*)dev(sizeof(int) * t);
    slices = (unsigned char*)dev((size_t)p * gst_vector_bytes(K.Dp));
    if (!slices || !K.CB) return HH_ENOMEM;
  } else {
    K.Wp = (double*)dev(sizeof(double) * t * 3 * D);
    if (!K.Wp) return HH_ENOMEM;
  }
  if (!K.Hpart || !K.azpart) return HH_ENOMEM;
  std::vector<double2*> vp(p);
  for (int a = 0; a < p; ++a) vp[a] = const_cast<double2*>(V) + (size_t)a * D;
  cudaMemcpyAsync(K.Vptr, vp.data(), sizeof(double2*) * p, cudaMemcpyHostToDevice, E.stream);
  const int pv = p;
  cudaMemcpyAsync(K.nV, &pv, sizeof(int), cudaMemcpyHostToDevice, E.stream);
  int rc;
  switch (t) {
    case 1: rc = gs_pass_t<1>(E, K, W, slices); break;
    case 2: rc = gs_pass_t<2>(E, K, W, slices); break;
    case 3: rc = gs_pass_t<3>(E, K, W, slices); break;
    default: rc = gs_pass_t<4>(E, K, W, slices); break;
  }
  if (rc) return rc;
  cudaMemcpyAsync(H_host, K.Hthis, sizeof(double2) * p * t, cudaMemcpyDeviceToHost, E.stream);
  cudaError_t e = cudaStreamSynchronize(E.stream);
  if (e != cudaSuccess) return (E.set_cuda_error(e, "Gram-Schmidt pass"), HH_ECUDA);
  return E.check_device_error("Gram-Schmidt pass");
}

}  // namespace hh
