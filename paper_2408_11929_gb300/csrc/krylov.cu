// Selective flexible multipreconditioned GMRES on the device (Section 3, selection rules of
// Section 4), FP64 complex.  Per iteration, for every active right-hand side r:
//   Z_k = [M_d^{-1} s_d]   (sweep.cu, all directions and right-hand sides in one launch)
//   W   = A Z_k            (matrix-free P1 stencil)
//   block CGS: H = V^H W, W -= V H, twice by default (opts.gs_passes), coefficients summed
//   block QR of W in preconditioner order (the same number of passes against the new vectors),
//     column j deflated when r_jj <= eta * ||w_j|| (norm after CGS2)
//   Givens update of the scalar upper Hessenberg matrix, rho = |g_last|, converged when
//     rho / ||b|| <= tol (tested once per iteration)
//   next sources: t = 1 the new vector, t = 2 the other preconditioner's new vector
//     ("cross"), t > 2 the normalised sum of the new vectors ("sum").
// At the end y = R^{-1} g, x = Z y and the explicit residual ||b - A x|| / ||b||.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "engine.h"

namespace hh {

void launch_pack(Engine& E, const double2* const* srcptr, const double* scale, int C, int t, int4 codes, void* X);
void launch_unpack(Engine& E, const void* X, int C, int t, int4 codes, double2* dst, size_t stride);

struct KState {
  int nrhs, t, D, maxit, maxV, maxZ, GX, GQ, scheme, passes;
  double tol, eta;
  double* beta;
  int *done, *status, *nV, *nZ, *iters, *nacc, *amap;
  double *rho, *nu, *cs, *hist, *npart;
  double2 **Vptr, **Zptr;
  double2 *Hacc, *Hthis, *Hpart, *Rnew, *sn, *g, *Rrot, *y, *qpart, *sbuf, *V0;
  const double2** srcptr;
  double* scale;
  double* res_exp;
};

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

// ------------------------------------------------------------------ operator
__global__ void spmv_kernel(const double2* __restrict__ x, double2* __restrict__ y, int ncols, Coef cf) {
  const int n = cf.n, m = n + 1;
  const size_t D = (size_t)m * m;
  const double dg = cf.diag();
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < D * ncols; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t c = idx / D, g = idx % D;
    const int j = (int)(g / m), i = (int)(g % m);
    const double2* xc = x + c * D;
    const int type = line_type(j, n);
    double2 acc = make_double2(0, 0);
    cfma(acc, cf.centre(i, type), xc[g]);
    const double2 hz = cf.horiz(type);
    if (i + 1 <= n) cfma(acc, hz, xc[g + 1]);
    if (i >= 1) cfma(acc, hz, xc[g - 1]);
    const double2 vt = cf.vert(i);
    if (j >= 1) {
      cfma(acc, vt, xc[g - m]);
      if (i >= 1) { const double2 v = xc[g - m - 1]; acc.x += dg * v.x; acc.y += dg * v.y; }
    }
    if (j + 1 <= n) {
      cfma(acc, vt, xc[g + m]);
      if (i + 1 <= n) { const double2 v = xc[g + m + 1]; acc.x += dg * v.x; acc.y += dg * v.y; }
    }
    y[idx] = acc;
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
__global__ void norm_part_kernel(const double2* __restrict__ x, size_t D, double* part, int GX) {
  const int r = blockIdx.y;
  const double2* xr = x + (size_t)r * D;
  double v[1] = {0};
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < D; g += (size_t)GX * blockDim.x) v[0] += cabs2(xr[g]);
  __shared__ double sh[32];
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) part[r * GX + blockIdx.x] = v[0];
}

__global__ void start_kernel(KState S, const double2* __restrict__ b) {
  const int r = blockIdx.x;
  if (threadIdx.x == 0) {
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

__global__ void scale_copy_kernel(KState S, const double2* __restrict__ b) {
  const int r = blockIdx.y;
  const double beta = S.beta[r];
  const double inv = beta > 0 ? 1.0 / beta : 0.0;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < (size_t)S.D; g += (size_t)gridDim.x * blockDim.x)
    S.V0[(size_t)r * S.D + g] = cscale(b[(size_t)r * S.D + g], inv);
}

// ------------------------------------------------------------------ Gram-Schmidt vs the basis
template <int TT, int AB>
__global__ void __launch_bounds__(256) gs_dot_kernel(KState S, const double2* __restrict__ W) {
  const int r = blockIdx.y;
  if (S.done[r]) return;
  const int nV = S.nV[r];
  const size_t D = S.D;
  const size_t chunk = (D + S.GX - 1) / S.GX;
  const size_t g0 = blockIdx.x * chunk, g1 = min(D, g0 + chunk);
  const double2* Wr = W + (size_t)r * TT * D;
  __shared__ double sh[32 * AB * TT * 2];
  for (int a0 = 0; a0 < nV; a0 += AB) {
    double acc[AB * TT * 2];
#pragma unroll
    for (int q = 0; q < AB * TT * 2; ++q) acc[q] = 0;
    const double2* vp[AB];
#pragma unroll
    for (int ab = 0; ab < AB; ++ab) vp[ab] = (a0 + ab < nV) ? S.Vptr[(size_t)r * S.maxV + a0 + ab] : nullptr;
    for (size_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
      double2 w[TT];
#pragma unroll
      for (int b = 0; b < TT; ++b) w[b] = Wr[b * D + g];
#pragma unroll
      for (int ab = 0; ab < AB; ++ab) {
        if (vp[ab]) {
          const double2 v = vp[ab][g];
#pragma unroll
          for (int b = 0; b < TT; ++b) {
            const int q = (ab * TT + b) * 2;
            acc[q] = fma(v.x, w[b].x, acc[q]); acc[q] = fma(v.y, w[b].y, acc[q]);
            acc[q + 1] = fma(v.x, w[b].y, acc[q + 1]); acc[q + 1] = fma(-v.y, w[b].x, acc[q + 1]);
          }
        }
      }
    }
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

__global__ void gs_reduce_kernel(KState S, int first) {
  const int r = blockIdx.x;
  if (S.done[r]) return;
  const int cnt = S.nV[r] * S.t;
  for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
    const size_t base = ((size_t)r * S.maxV * S.t + p);
    double2 s = make_double2(0, 0);
    for (int q = 0; q < S.GX; ++q) s = cadd(s, S.Hpart[base * S.GX + q]);
    S.Hthis[base] = s;
    S.Hacc[base] = first ? s : cadd(S.Hacc[base], s);
  }
}

template <int TT>
__global__ void __launch_bounds__(256) gs_update_kernel(KState S, double2* __restrict__ W) {
  const int r = blockIdx.y;
  if (S.done[r]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nV = S.nV[r];
  double2* Hs = reinterpret_cast<double2*>(smem_raw);
  const double2** vps = reinterpret_cast<const double2**>(Hs + (size_t)nV * TT);
  for (int p = threadIdx.x; p < nV * TT; p += blockDim.x) Hs[p] = S.Hthis[(size_t)r * S.maxV * TT + p];
  for (int a = threadIdx.x; a < nV; a += blockDim.x) vps[a] = S.Vptr[(size_t)r * S.maxV + a];
  __syncthreads();
  const size_t D = S.D;
  double2* Wr = W + (size_t)r * TT * D;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < D; g += (size_t)gridDim.x * blockDim.x) {
    double2 w[TT];
#pragma unroll
    for (int b = 0; b < TT; ++b) w[b] = Wr[b * D + g];
    for (int a = 0; a < nV; ++a) {
      const double2 v = vps[a][g];
#pragma unroll
      for (int b = 0; b < TT; ++b) {
        const double2 hh = Hs[a * TT + b];
        w[b].x = fma(-v.x, hh.x, w[b].x); w[b].x = fma(v.y, hh.y, w[b].x);
        w[b].y = fma(-v.x, hh.y, w[b].y); w[b].y = fma(-v.y, hh.x, w[b].y);
      }
    }
#pragma unroll
    for (int b = 0; b < TT; ++b) Wr[b * D + g] = w[b];
  }
}

// ------------------------------------------------------------------ block QR (cooperative)
// Grid (GQ, nrhs).  Every reduction: per-CTA partials into qpart[parity], grid barrier,
// every CTA of the right-hand side sums the GQ partials in the same order (so all take the
// same deflation decisions).  The barrier sequence is the same for every CTA.
template <int TT>
__global__ void __launch_bounds__(256) qr_kernel(KState S, double2* __restrict__ W, double2* __restrict__ Vk,
                                                 unsigned* bar, int* err, long long budget) {
  const int r = blockIdx.y;
  const bool active = S.done[r] == 0;
  const size_t D = S.D;
  const size_t chunk = (D + S.GQ - 1) / S.GQ;
  const size_t g0 = blockIdx.x * chunk, g1 = min(D, g0 + chunk);
  double2* Wr = W + (size_t)r * TT * D;
  double2* Vr = Vk + (size_t)r * TT * D;
  __shared__ double sh[32 * 8];
  __shared__ double2 red_out[TT];
  unsigned target = 0;
  int parity = 0;
  const bool writer = blockIdx.x == 0 && threadIdx.x == 0;
  if (writer && active)
    for (int q = 0; q < TT * TT; ++q) S.Rnew[(size_t)r * TT * TT + q] = make_double2(0, 0);

  // reduce TT complex values (in v[2*TT]) across the CTAs of this right-hand side
  auto reduce = [&](double (&v)[2 * TT]) -> bool {
    block_sum<2 * TT>(v, sh);
    double2* part = S.qpart + ((size_t)parity * S.nrhs + r) * S.GQ * TT;
    if (threadIdx.x == 0)
      for (int q = 0; q < TT; ++q) part[(size_t)blockIdx.x * TT + q] = make_double2(v[2 * q], v[2 * q + 1]);
    if (!grid_sync(bar, target, err, budget)) return false;
    if (threadIdx.x == 0) {
      for (int q = 0; q < TT; ++q) {
        double2 s = make_double2(0, 0);
        for (int b = 0; b < S.GQ; ++b) s = cadd(s, __ldcg(part + (size_t)b * TT + q));
        red_out[q] = s;
      }
    }
    __syncthreads();
    parity ^= 1;
    return true;
  };

  double nu[TT];
  {
    double v[2 * TT];
    for (int q = 0; q < 2 * TT; ++q) v[q] = 0;
    if (active)
      for (size_t g = g0 + threadIdx.x; g < g1; g += blockDim.x)
#pragma unroll
        for (int j = 0; j < TT; ++j) v[2 * j] += cabs2(Wr[j * D + g]);
    if (!reduce(v)) return;
    for (int j = 0; j < TT; ++j) nu[j] = sqrt(red_out[j].x);
  }
  int acc = 0;
  int amap[TT];
  for (int j = 0; j < TT; ++j) {
    double2* w = Wr + j * D;
    for (int pass = 0; pass < S.passes; ++pass) {
      double v[2 * TT];
      for (int q = 0; q < 2 * TT; ++q) v[q] = 0;
      if (active && acc > 0)
        for (size_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
          const double2 wv = w[g];
          for (int q = 0; q < acc; ++q) {
            const double2 vq = Vr[q * D + g];
            v[2 * q] = fma(vq.x, wv.x, v[2 * q]); v[2 * q] = fma(vq.y, wv.y, v[2 * q]);
            v[2 * q + 1] = fma(vq.x, wv.y, v[2 * q + 1]); v[2 * q + 1] = fma(-vq.y, wv.x, v[2 * q + 1]);
          }
        }
      if (!reduce(v)) return;
      if (active && acc > 0) {
        double2 c[TT];
        for (int q = 0; q < TT; ++q) c[q] = red_out[q];
        for (size_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
          double2 wv = w[g];
          for (int q = 0; q < acc; ++q) wv = csub(wv, cmul(c[q], Vr[q * D + g]));
          w[g] = wv;
        }
        if (writer)
          for (int q = 0; q < acc; ++q) {
            double2* p = S.Rnew + (size_t)r * TT * TT + q * TT + j;
            *p = cadd(*p, c[q]);
          }
      }
      __syncthreads();
    }
    double v[2 * TT];
    for (int q = 0; q < 2 * TT; ++q) v[q] = 0;
    if (active)
      for (size_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) v[0] += cabs2(w[g]);
    if (!reduce(v)) return;
    const double rjj = sqrt(red_out[0].x);
    amap[j] = -1;
    if (active && rjj > S.eta * nu[j] && rjj > 0 && isfinite(rjj)) {
      const double inv = 1.0 / rjj;
      double2* vo = Vr + acc * D;
      for (size_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) vo[g] = cscale(w[g], inv);
      if (writer) S.Rnew[(size_t)r * TT * TT + acc * TT + j] = make_double2(rjj, 0);
      amap[j] = acc;
      ++acc;
    }
    __syncthreads();
  }
  if (writer && active) {
    S.nacc[r] = acc;
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

__global__ void hess_kernel(KState S, double2* __restrict__ Zk, double2* __restrict__ Vk) {
  const int r = blockIdx.x;
  if (threadIdx.x != 0 || S.done[r]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* col = reinterpret_cast<double2*>(smem_raw);
  const int t = S.t;
  const int nold = S.nV[r], nacc = S.nacc[r];
  const size_t D = S.D;
  double2* g = S.g + (size_t)r * (S.maxZ + 1);
  if (nacc == 0) {
    S.status[r] = HH_EBREAKDOWN;
    S.done[r] = 1;
    return;
  }
  int nZ = S.nZ[r];
  for (int j = 0; j < t; ++j) {
    const int pos = S.amap[r * t + j];
    if (pos < 0) continue;
    const int c = nZ;
    const int len = nold + pos + 1;  // == c + 2
    for (int i = 0; i < nold; ++i) col[i] = S.Hacc[((size_t)r * S.maxV + i) * t + j];
    for (int q = 0; q <= pos; ++q) col[nold + q] = S.Rnew[(size_t)r * t * t + q * t + j];
    for (int i = len; i < c + 2; ++i) col[i] = make_double2(0, 0);
    for (int i = 0; i < c; ++i) {
      const double cs = S.cs[(size_t)r * S.maxZ + i];
      const double2 sn = S.sn[(size_t)r * S.maxZ + i];
      const double2 a0 = col[i], a1 = col[i + 1];
      col[i] = cadd(cscale(a0, cs), cmul(sn, a1));
      const double2 msc = make_double2(-sn.x, sn.y);  // -conj(sn)
      col[i + 1] = cadd(cmul(msc, a0), cscale(a1, cs));
    }
    double cs;
    double2 sn;
    givens(col[c], col[c + 1], cs, sn);
    col[c] = cadd(cscale(col[c], cs), cmul(sn, col[c + 1]));
    S.cs[(size_t)r * S.maxZ + c] = cs;
    S.sn[(size_t)r * S.maxZ + c] = sn;
    double2* Rc = S.Rrot + (size_t)r * ((size_t)S.maxZ * (S.maxZ + 1) / 2) + (size_t)c * (c + 1) / 2;
    for (int i = 0; i <= c; ++i) Rc[i] = col[i];
    const double2 g0 = g[c];
    g[c] = cscale(g0, cs);
    g[c + 1] = cmul(make_double2(-sn.x, sn.y), g0);
    S.Zptr[(size_t)r * S.maxZ + c] = Zk + ((size_t)r * t + j) * D;
    nZ = c + 1;
  }
  for (int q = 0; q < nacc; ++q) S.Vptr[(size_t)r * S.maxV + nold + q] = Vk + ((size_t)r * t + q) * D;
  S.nV[r] = nold + nacc;
  S.nZ[r] = nZ;
  const int it = S.iters[r] + 1;
  S.iters[r] = it;
  const double rho = sqrt(cabs2(g[nZ]));
  S.rho[r] = rho;
  S.hist[(size_t)r * S.maxit + it - 1] = rho / S.beta[r];
  if (!isfinite(rho)) { S.status[r] = HH_ENAN; S.done[r] = 1; }
  else if (rho / S.beta[r] <= S.tol) { S.status[r] = HH_OK; S.done[r] = 1; }
  else if (it >= S.maxit) { S.status[r] = HH_ENOCONV; S.done[r] = 1; }
}

// next sources: sum of the new vectors (t > 2), with its norm
__global__ void source_sum_kernel(KState S, const double2* __restrict__ Vk) {
  const int r = blockIdx.y;
  if (S.done[r] || S.scheme != HH_SCHEME_SUM) return;
  const int nacc = S.nacc[r];
  const size_t D = S.D;
  const double2* Vr = Vk + (size_t)r * S.t * D;
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

__global__ void source_final_kernel(KState S, const double2* __restrict__ Vk) {
  const int r = blockIdx.x;
  if (threadIdx.x != 0 || S.done[r]) return;
  const int t = S.t;
  const size_t D = S.D;
  const double2* Vr = Vk + (size_t)r * t * D;
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
__global__ void backsub_kernel(KState S) {
  const int r = blockIdx.x;
  if (threadIdx.x != 0) return;
  const int nZ = S.nZ[r];
  const double2* Rb = S.Rrot + (size_t)r * ((size_t)S.maxZ * (S.maxZ + 1) / 2);
  const double2* g = S.g + (size_t)r * (S.maxZ + 1);
  double2* y = S.y + (size_t)r * S.maxZ;
  for (int i = nZ - 1; i >= 0; --i) {
    double2 s = g[i];
    for (int c = i + 1; c < nZ; ++c) s = csub(s, cmul(Rb[(size_t)c * (c + 1) / 2 + i], y[c]));
    const double2 d = Rb[(size_t)i * (i + 1) / 2 + i];
    const double dd = cabs2(d);
    y[i] = cmul(s, make_double2(d.x / dd, -d.y / dd));
  }
}

__global__ void xsol_kernel(KState S, double2* __restrict__ x) {
  const int r = blockIdx.y;
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
    x[(size_t)r * D + g] = a;
  }
}

__global__ void resid_part_kernel(const double2* __restrict__ b, const double2* __restrict__ Ax, size_t D,
                                  double* part, int GX) {
  const int r = blockIdx.y;
  double v[1] = {0};
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < D; g += (size_t)GX * blockDim.x) {
    const double2 d = csub(b[(size_t)r * D + g], Ax[(size_t)r * D + g]);
    v[0] += cabs2(d);
  }
  __shared__ double sh[32];
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) part[r * GX + blockIdx.x] = v[0];
}

__global__ void resid_final_kernel(KState S) {
  const int r = blockIdx.x;
  if (threadIdx.x != 0) return;
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

// ------------------------------------------------------------------ host driver
namespace {
struct DevBuf {
  Engine* E = nullptr;
  std::vector<void*> ptrs;
  template <typename T> T* get(size_t count) {
    void* p = nullptr;
    if (E->dmalloc(&p, std::max<size_t>(count * sizeof(T), 16))) return nullptr;
    cudaMemsetAsync(p, 0, std::max<size_t>(count * sizeof(T), 16), E->stream);
    ptrs.push_back(p);
    return reinterpret_cast<T*>(p);
  }
  ~DevBuf() {
    for (void* p : ptrs) E->dfree(p);
  }
};
}  // namespace

template <int TT>
static void launch_iteration_gs(Engine& E, KState& S, double2* W, dim3 gsgrid) {
  for (int pass = 0; pass < S.passes; ++pass) {
    gs_dot_kernel<TT, 4><<<gsgrid, 256, 0, E.stream>>>(S, W);
    gs_reduce_kernel<<<S.nrhs, 256, 0, E.stream>>>(S, pass == 0);
    const size_t smem = (size_t)S.maxV * TT * sizeof(double2) + (size_t)S.maxV * sizeof(void*);
    cudaFuncSetAttribute((const void*)gs_update_kernel<TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    gs_update_kernel<TT><<<gsgrid, 256, smem, E.stream>>>(S, W);
    E.count_launch(3);
  }
}

template <int TT>
static cudaError_t launch_qr(Engine& E, KState& S, double2* W, double2* Vk) {
  cudaMemsetAsync(E.bar, 0, sizeof(unsigned), E.stream);
  void* args[] = {(void*)&S, (void*)&W, (void*)&Vk, (void*)&E.bar, (void*)&E.err, (void*)&E.opts.timeout_cycles};
  return E.launch_coop((const void*)qr_kernel<TT>, S.GQ, 256, 0, args, S.nrhs);
}

int Engine::solve_batch_dev(int nrhs, const double2* b, double2* x, double tol, hh_result* res) {
  const int maxit = opts.maxit;
  const size_t D = (size_t)m * m;
  KState S{};
  S.nrhs = nrhs; S.t = t; S.D = (int)D; S.maxit = maxit; S.maxV = 1 + maxit * t; S.maxZ = maxit * t;
  S.tol = tol; S.eta = opts.deflate_eta; S.passes = opts.gs_passes;
  S.scheme = opts.scheme != HH_SCHEME_AUTO ? opts.scheme : (t == 2 ? HH_SCHEME_CROSS : (t > 2 ? HH_SCHEME_SUM : HH_SCHEME_CROSS));
  S.GX = std::max(1, std::min(num_sms * 2 / std::max(1, nrhs) + 1, (int)((D + 255) / 256)));
  S.GX = std::min(S.GX, num_sms * 2);
  {
    int per_sm = coop_per_sm;
    int cap = num_sms * per_sm;
    S.GQ = std::max(1, std::min(cap / nrhs, num_sms));
    if (S.GQ * nrhs > cap) return (set_error("too many right-hand sides for one cooperative QR launch"), HH_EINVAL);
  }
  DevBuf B;
  B.E = this;
  S.beta = B.get<double>(nrhs); S.done = B.get<int>(nrhs); S.status = B.get<int>(nrhs);
  S.nV = B.get<int>(nrhs); S.nZ = B.get<int>(nrhs); S.iters = B.get<int>(nrhs); S.nacc = B.get<int>(nrhs);
  S.amap = B.get<int>((size_t)nrhs * t); S.rho = B.get<double>(nrhs); S.nu = B.get<double>((size_t)nrhs * t);
  S.cs = B.get<double>((size_t)nrhs * S.maxZ); S.sn = B.get<double2>((size_t)nrhs * S.maxZ);
  S.hist = B.get<double>((size_t)nrhs * maxit); S.npart = B.get<double>((size_t)nrhs * S.GX);
  S.Vptr = B.get<double2*>((size_t)nrhs * S.maxV); S.Zptr = B.get<double2*>((size_t)nrhs * S.maxZ);
  S.Hacc = B.get<double2>((size_t)nrhs * S.maxV * t); S.Hthis = B.get<double2>((size_t)nrhs * S.maxV * t);
  S.Hpart = B.get<double2>((size_t)nrhs * S.maxV * t * S.GX); S.Rnew = B.get<double2>((size_t)nrhs * t * t);
  S.g = B.get<double2>((size_t)nrhs * (S.maxZ + 1));
  S.Rrot = B.get<double2>((size_t)nrhs * ((size_t)S.maxZ * (S.maxZ + 1) / 2));
  S.y = B.get<double2>((size_t)nrhs * S.maxZ); S.qpart = B.get<double2>((size_t)2 * nrhs * S.GQ * 4);
  S.sbuf = B.get<double2>((size_t)nrhs * D); S.V0 = B.get<double2>((size_t)nrhs * D);
  S.srcptr = (const double2**)B.get<double2*>((size_t)nrhs * t); S.scale = B.get<double>((size_t)nrhs * t);
  S.res_exp = B.get<double>(nrhs);
  double2* W = B.get<double2>((size_t)nrhs * t * D);
  if (!W || !S.res_exp || !S.V0 || !S.Rrot) return HH_ENOMEM;
  const int C = nrhs * t;
  if (ensure_sweep_ws(C)) return HH_ENOMEM;
  int4 codes = make_int4(0, 0, 0, 0);
  int* cp = &codes.x;
  for (int d = 0; d < t; ++d) cp[d] = dir_codes[d];

  // beta, V0
  dim3 ng(S.GX, nrhs);
  norm_part_kernel<<<ng, 256, 0, stream>>>(b, D, S.npart, S.GX);
  start_kernel<<<nrhs, 32, 0, stream>>>(S, b);
  scale_copy_kernel<<<ng, 256, 0, stream>>>(S, b);
  count_launch(3);

  std::vector<double2*> zblocks, vblocks;
  std::vector<int> h_done(nrhs), h_status(nrhs), h_iters(nrhs);
  int* pinned_done = nullptr;
  cudaMallocHost((void**)&pinned_done, sizeof(int) * nrhs);
  int rc = HH_OK;
  int k = 0;
  for (k = 1; k <= maxit; ++k) {
    double2 *Zk = nullptr, *Vk = nullptr;
    if (dmalloc((void**)&Zk, (size_t)C * D * sizeof(double2)) || dmalloc((void**)&Vk, (size_t)C * D * sizeof(double2))) {
      dfree(Zk);
      rc = HH_ENOMEM;
      break;
    }
    zblocks.push_back(Zk);
    vblocks.push_back(Vk);
    // preconditioners: every (rhs, direction) pair is one sweep column
    launch_pack(*this, S.srcptr, S.scale, C, t, codes, w_rin);
    rc = run_sweep(w_rin, w_v, w_w, C, opts.single_sweep != 0);
    if (rc) break;
    launch_unpack(*this, w_v, C, t, codes, Zk, D);
    // W = A Z_k
    tick_begin(K_SPMV);
    spmv_kernel<<<grid_for(D * C), 256, 0, stream>>>(Zk, W, C, coef);
    count_launch();
    tick_end(K_SPMV, 2.0 * C * D * 16.0, 0);
    // Gram-Schmidt
    tick_begin(K_GS);
    dim3 gsgrid(S.GX, nrhs);
    switch (t) {
      case 1: launch_iteration_gs<1>(*this, S, W, gsgrid); break;
      case 2: launch_iteration_gs<2>(*this, S, W, gsgrid); break;
      case 3: launch_iteration_gs<3>(*this, S, W, gsgrid); break;
      default: launch_iteration_gs<4>(*this, S, W, gsgrid); break;
    }
    cudaError_t ce;
    switch (t) {
      case 1: ce = launch_qr<1>(*this, S, W, Vk); break;
      case 2: ce = launch_qr<2>(*this, S, W, Vk); break;
      case 3: ce = launch_qr<3>(*this, S, W, Vk); break;
      default: ce = launch_qr<4>(*this, S, W, Vk); break;
    }
    {
      // algorithmic bytes of Gram-Schmidt this iteration: two passes of (read V + read W)
      // for the dot products and (read V + read/write W) for the update, plus the block QR
      const double nVmax = 1.0 + (double)(k - 1) * t;
      tick_end(K_GS, nrhs * (S.passes * (2.0 * nVmax * D * 16 + 3.0 * t * D * 16) + 6.0 * t * D * 16), 0);
    }
    if (ce != cudaSuccess) { set_cuda_error(ce, "qr launch"); rc = HH_ECUDA; break; }
    const size_t hsmem = (size_t)(S.maxZ + 2) * sizeof(double2);
    cudaFuncSetAttribute((const void*)hess_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem);
    hess_kernel<<<nrhs, 32, hsmem, stream>>>(S, Zk, Vk);
    source_sum_kernel<<<ng, 256, 0, stream>>>(S, Vk);
    source_final_kernel<<<nrhs, 32, 0, stream>>>(S, Vk);
    count_launch(4);
    cudaMemcpyAsync(pinned_done, S.done, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, stream);
    cudaError_t se = cudaStreamSynchronize(stream);
    if (se != cudaSuccess) { set_cuda_error(se, "iteration"); rc = HH_ECUDA; break; }
    rc = check_device_error("iteration");
    if (rc) break;
    bool all = true;
    for (int r = 0; r < nrhs; ++r) all = all && pinned_done[r];
    if (all) break;
  }
  if (rc == HH_OK) {
    backsub_kernel<<<nrhs, 32, 0, stream>>>(S);
    const size_t xsmem = (size_t)S.maxZ * (sizeof(double2) + sizeof(void*));
    cudaFuncSetAttribute((const void*)xsol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsmem);
    xsol_kernel<<<dim3(S.GX, nrhs), 256, xsmem, stream>>>(S, x);
    tick_begin(K_SPMV);
    spmv_kernel<<<grid_for(D * nrhs), 256, 0, stream>>>(x, W, nrhs, coef);
    tick_end(K_SPMV, 2.0 * nrhs * D * 16.0, 0);
    resid_part_kernel<<<ng, 256, 0, stream>>>(b, W, D, S.npart, S.GX);
    resid_final_kernel<<<nrhs, 32, 0, stream>>>(S);
    count_launch(5);
    std::vector<double> h_rho(nrhs), h_beta(nrhs), h_res(nrhs);
    cudaMemcpyAsync(h_status.data(), S.status, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, stream);
    cudaMemcpyAsync(h_iters.data(), S.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, stream);
    cudaMemcpyAsync(h_rho.data(), S.rho, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, stream);
    cudaMemcpyAsync(h_beta.data(), S.beta, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, stream);
    cudaMemcpyAsync(h_res.data(), S.res_exp, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, stream);
    cudaError_t se = cudaStreamSynchronize(stream);
    if (se != cudaSuccess) { set_cuda_error(se, "final"); rc = HH_ECUDA; }
    int worst = HH_OK;
    for (int r = 0; r < nrhs && rc == HH_OK; ++r) {
      if (res) {
        res[r].iterations = h_iters[r];
        res[r].rel_res_implicit = h_beta[r] > 0 ? h_rho[r] / h_beta[r] : 0.0;
        res[r].rel_res_explicit = h_res[r];
        res[r].status = (hh_status)h_status[r];
      }
      if (h_status[r] != HH_OK && worst == HH_OK) worst = h_status[r];
    }
    if (rc == HH_OK) rc = worst;
  }
  cudaStreamSynchronize(stream);
  for (auto p : zblocks) dfree(p);
  for (auto p : vblocks) dfree(p);
  cudaFreeHost(pinned_done);
  collect_ticks();
  return rc;
}

int Engine::apply_operator(int ncols, const double2* x, double2* y) {
  const size_t D = (size_t)m * m;
  tick_begin(K_SPMV);
  spmv_kernel<<<grid_for(D * ncols), 256, 0, stream>>>(x, y, ncols, coef);
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
  gauss_nodal_kernel<<<grid_for(D), 256, 0, stream>>>(dsrc, nsrc, n, f);
  mass_neg_kernel<<<grid_for(D), 256, 0, stream>>>(f, rhs, n);
  count_launch(2);
  cudaError_t e = cudaStreamSynchronize(stream);
  dfree(dsrc);
  dfree(f);
  if (e != cudaSuccess) { set_cuda_error(e, "assemble_rhs"); return HH_ECUDA; }
  return HH_OK;
}

int Engine::apply_preconditioner_dev(int dcode, int ncols, const double2* r, double2* z, bool single) {
  const size_t D = (size_t)m * m;
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
