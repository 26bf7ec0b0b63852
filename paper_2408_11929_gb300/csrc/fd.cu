// The paper's own discretisation and decomposition (Section 4) as a mode of the engine
// (hh_opts.discretization = HH_DISC_FD): five-point finite differences on the uniform grid
// and N overlapping strips whose double sweeps exchange Robin data (Section 2, Eqs. (2)-(4)),
// FP64 on the CUDA cores.
//
// Discretisation (the same readings as the oracle's FD mode): interior rows (4 - k^2 h^2) u -
// (four neighbours); a Robin side of a node has a ghost node, eliminated with the centred
// difference of du/dn - i k u = g, so the inward neighbour's coefficient doubles and the centre
// gains -2 i k h; a row is scaled by 1/2 per boundary side (complex symmetric matrix).
//
// Decomposition: strip s holds cell layers sR..(s+1)R and owns node lines
// a_s = max(0, sR - 1) .. b_s = min(n, (s+1)R + 1) (neighbours overlap by three lines, 2h).
// The subdomain problem is the same five-point Robin problem on its rectangle: its matrix
// depends only on its line count L, and is block tridiagonal over the lines with
//   D_l = tridiagonal line operator (boundary type for l = 0 and l = L-1, else interior),
//   L_l = U_l = -diag(s_i)  (s_i = 1/2 at i = 0, n, else 1; the doubled inward coupling of a
//                            boundary line times its row scale 1/2 is again -s_i),
// so block Thomas needs S_0 = D_bnd, S_l = D_int - diag(s) S_{l-1}^{-1} diag(s) and the top
// S_{L-1} = D_bnd - diag(s) S_{L-2}^{-1} diag(s): one chain of inverses F_l = S_l^{-1} serves
// every subdomain, plus one top inverse per distinct L (first and last strip: L = R+2,
// interior strips: L = R+3).  Inverses by Gauss-Jordan with partial pivoting (setup.cu).
//
// Sweep of one direction (in its frame: lines counted in the sweep direction, Section 4's
// four directions are relabellings of the bottom-to-top sweep): forward s = 0..N-1, v_s with
// the Robin data of v_{s-1} on its lower artificial line; backward s = N-2..0, u_s with the
// data of v_{s-1} below and of u_{s+1} above (u_{N-1} = v_{N-1}); the right-hand side of a
// subdomain is the residual rescaled from the global rows' scales to the subdomain's plus
// s_sub 2h B(w) on an artificial line, B(w) = dw/dn - i k w by the centred difference.  Every
// node of the output takes the most recent subdomain solve that contains it.  All t
// directions and right-hand sides are columns of one sweep.
#include <algorithm>
#include <cmath>
#include <functional>
#include <vector>

#include "common.cuh"
#include "engine.h"

namespace hh {

// setup.cu: out[q] = S_q^{-1} (complex128, pivoted Gauss-Jordan), S_q formed by form(q, S)
// into a scratch block just before its inversion (it may read the earlier inverses)
int invert_chain_fp64(Engine& E, int count, const std::function<int(int, double2*)>& form, double2* const* out);

struct FdState {
  int Lmax = 0;                 // lines of the largest subdomain
  std::vector<int> a, L;        // per strip: first frame line, line count
  int nchain = 0;               // chain inverses F_0 .. F_{nchain-1}
  std::vector<int> tops;        // distinct line counts; the top inverse of tops[q] is block nchain + q
  double2* F = nullptr;         // inverses, m x ldf each
  int nblk = 0;
  int Cmax = 0;
  double2 *X = nullptr, *Y = nullptr, *sub = nullptr, *fbuf = nullptr;
};

static __host__ __device__ __forceinline__ double fd_s(int i, int n) { return (i == 0 || i == n) ? 0.5 : 1.0; }

// ------------------------------------------------------------------ setup kernels
// dense m x m line block: boundary = 1 for a line on the rectangle's boundary (row scale 1/2 and
// one more Robin side), 0 for an interior line
__global__ void fd_line_block_kernel(double2* __restrict__ D, int n, int ld, double k, int boundary) {
  const int m = n + 1;
  const double h = 1.0 / n, kh2 = k * k * h * h, kh = k * h;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)m * m; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    const double s = fd_s(i, n) * (boundary ? 0.5 : 1.0);
    const int nsides = (i == 0 || i == n) + boundary;
    double2 v = make_double2(0, 0);
    if (j == i) {
      v = make_double2(s * (4.0 - kh2), -s * 2.0 * kh * nsides);
    } else if (j == i + 1 || j == i - 1) {
      // the ghost beyond i = 0 (i = n) is the mirror of i + 1 (i - 1): that coupling doubles
      const bool doubled = (i == 0) || (i == n);
      v = make_double2(-s * (doubled ? 2.0 : 1.0), 0);
    }
    D[(size_t)i * ld + j] = v;
  }
}

// S = D - diag(s) Fprev diag(s)  (Fprev may be null: S = D)
__global__ void fd_schur_kernel(const double2* __restrict__ D, const double2* __restrict__ Fprev,
                                double2* __restrict__ S, int n, int ld) {
  const int m = n + 1;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)m * m; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    double2 v = D[(size_t)i * ld + j];
    if (Fprev) {
      const double w = fd_s(i, n) * fd_s(j, n);
      const double2 f = Fprev[(size_t)i * ld + j];
      v.x -= w * f.x;
      v.y -= w * f.y;
    }
    S[(size_t)i * ld + j] = v;
  }
}

// ------------------------------------------------------------------ sweep kernels
// Frame of a direction code (lines counted in the sweep direction): frame node (l, i) is grid
// node (gi, gj) with BT: (i, l), TB: (i, n - l), LR: (l, i), RL: (n - l, i).
__device__ __forceinline__ size_t fd_global(int code, int l, int i, int n) {
  int gi, gj;
  switch (code) {
    case DC_BT: gi = i; gj = l; break;
    case DC_TB: gi = i; gj = n - l; break;
    case DC_LR: gi = l; gj = i; break;
    default: gi = n - l; gj = i; break;  // DC_RL
  }
  return (size_t)gj * (n + 1) + gi;
}

__device__ __forceinline__ int code_of(int4 codes, int d) {
  return d == 0 ? codes.x : d == 1 ? codes.y : d == 2 ? codes.z : codes.w;
}

// X[(l m + i) C + c] = scale[c] src[c][global(l, i)], column c in direction codes[c % t]
__global__ void fd_pack_kernel(const double2* const* __restrict__ src, const double* __restrict__ scale, int C,
                               int t, int4 codes, double2* __restrict__ X, int n) {
  const size_t m = n + 1;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < m * m * C; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const size_t node = e / C;
    const int l = (int)(node / m), i = (int)(node % m);
    const double2 v = src[c][fd_global(code_of(codes, c % t), l, i, n)];
    const double sc = scale ? scale[c] : 1.0;
    X[e] = make_double2(sc * v.x, sc * v.y);
  }
}

__global__ void fd_unpack_kernel(const double2* __restrict__ Y, double2* const* __restrict__ dst, int C, int t,
                                 int4 codes, int n) {
  const size_t m = n + 1;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < m * m * C; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const size_t node = e / C;
    const int l = (int)(node / m), i = (int)(node % m);
    dst[c][fd_global(code_of(codes, c % t), l, i, n)] = Y[e];
  }
}

// Right-hand side of a subdomain (lines a .. a + L - 1 of the frame): the residual rescaled
// from the global rows' line scale to the subdomain's, plus s_sub 2h B(w) on an artificial
// line, B(w) = dw/dn - i k w by the centred difference over w's lines p - 1, p, p + 1.
// lo / hi: the neighbour's solution (its first frame line lo_a / hi_a), or null.
__global__ void fd_rhs_kernel(const double2* __restrict__ X, double2* __restrict__ f, int a, int L,
                              const double2* __restrict__ lo, int lo_a, const double2* __restrict__ hi, int hi_a,
                              int n, int C, double k) {
  const size_t m = n + 1, line = m * C;
  const double h = 1.0 / n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)L * line; e += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(e / line);
    const size_t rest = e % line;  // i C + c
    const int i = (int)(rest / C);
    const int gl = a + l;
    const double ratio = ((l == 0 || l == L - 1) ? 0.5 : 1.0) / ((gl == 0 || gl == n) ? 0.5 : 1.0);
    const double2 x = X[(size_t)gl * line + rest];
    double2 v = make_double2(ratio * x.x, ratio * x.y);
    const double wdata = fd_s(i, n) * 0.5 * 2.0 * h;  // s_sub 2h on a boundary line
    if (l == 0 && lo) {
      // outward normal towards lower lines: dw/dn = (w[p-1] - w[p+1]) / 2h
      const int p = a - lo_a;
      const double2 wm = lo[(size_t)(p - 1) * line + rest], w0 = lo[(size_t)p * line + rest];
      const double2 wp = lo[(size_t)(p + 1) * line + rest];
      const double2 g = make_double2((wm.x - wp.x) / (2.0 * h) + k * w0.y, (wm.y - wp.y) / (2.0 * h) - k * w0.x);
      v.x += wdata * g.x;
      v.y += wdata * g.y;
    }
    if (l == L - 1 && hi) {
      const int p = a + L - 1 - hi_a;
      const double2 wm = hi[(size_t)(p - 1) * line + rest], w0 = hi[(size_t)p * line + rest];
      const double2 wp = hi[(size_t)(p + 1) * line + rest];
      const double2 g = make_double2((wp.x - wm.x) / (2.0 * h) + k * w0.y, (wp.y - wm.y) / (2.0 * h) - k * w0.x);
      v.x += wdata * g.x;
      v.y += wdata * g.y;
    }
    f[e] = v;
  }
}

// out[r][c] = base[r][c] + sum_k F[r][k] (a[k][c] + s_k b[k][c]) for one node line (rows r of
// the m x m inverse F); a, b, base may be null.  The input line is staged in shared memory as
// the three planes of Gauss's complex product (Re v, Im v - Re v, Re v + Im v), so that each
// complex multiply-add is three FP64 FMAs; a warp per row, lanes over k.
constexpr int FD_ROWS = 4;  // rows (warps) per CTA
__host__ __device__ constexpr size_t fd_step_smem(int m, int C) { return (size_t)m * C * 3 * sizeof(double); }
__global__ void __launch_bounds__(32 * FD_ROWS) fd_step_kernel(const double2* __restrict__ F, int ld,
                                                               const double2* __restrict__ a,
                                                               const double2* __restrict__ b,
                                                               const double2* base, double2* out, int n, int C) {
  extern __shared__ __align__(16) unsigned char fd_smem[];
  double* x = reinterpret_cast<double*>(fd_smem);  // m x C x 3
  const int m = n + 1;
  for (int e = threadIdx.x; e < m * C; e += blockDim.x) {
    const int kk = e / C;
    double2 v = a ? a[e] : make_double2(0, 0);
    if (b) {
      const double s = fd_s(kk, n);
      const double2 w = b[e];
      v.x += s * w.x;
      v.y += s * w.y;
    }
    x[3 * e] = v.x;
    x[3 * e + 1] = v.y - v.x;
    x[3 * e + 2] = v.x + v.y;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * FD_ROWS + (threadIdx.x >> 5);
  if (r >= m) return;
  constexpr int CM = 8;  // columns per pass
  const double2* Fr = F + (size_t)r * ld;
  for (int c0 = 0; c0 < C; c0 += CM) {
    double p1[CM], p2[CM], p3[CM];
#pragma unroll
    for (int q = 0; q < CM; ++q) p1[q] = p2[q] = p3[q] = 0;
    for (int kk = lane; kk < m; kk += 32) {
      const double2 f = Fr[kk];
      const double fs = f.x + f.y;
#pragma unroll
      for (int q = 0; q < CM; ++q) {
        if (c0 + q < C) {
          const double* v = x + 3 * ((size_t)kk * C + c0 + q);
          // (f.x + i f.y)(v.x + i v.y): re = fs v.x - f.y (v.x + v.y), im = fs v.x + f.x (v.y - v.x)
          p1[q] = fma(fs, v[0], p1[q]);
          p2[q] = fma(f.x, v[1], p2[q]);
          p3[q] = fma(f.y, v[2], p3[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < CM; ++q) {
      double re = p1[q] - p3[q], im = p1[q] + p2[q];
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane == 0 && c0 + q < C) {
        const size_t idx = (size_t)r * C + c0 + q;
        double2 o = base ? base[idx] : make_double2(0, 0);
        o.x += re;
        o.y += im;
        out[idx] = o;
      }
    }
  }
}

// Y lines a .. a + L - 1 = the subdomain's solution (the caller orders the copies so that the
// most recent solve of an overlap is written last)
__global__ void fd_place_kernel(const double2* __restrict__ sub, double2* __restrict__ Y, int a, int L, int n, int C) {
  const size_t line = (size_t)(n + 1) * C;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)L * line; e += (size_t)gridDim.x * blockDim.x)
    Y[(size_t)a * line + e] = sub[e];
}

// y = A x, five-point Robin operator with row scaling, natural node order g = j m + i
__global__ void fd_operator_kernel(const double2* const* __restrict__ xcol, double2* const* __restrict__ ycol,
                                   int ncols, int n, double k) {
  const int c = blockIdx.y;
  const int m = n + 1;
  const double h = 1.0 / n, kh2 = k * k * h * h, kh = k * h;
  const double2* x = xcol[c];
  double2* y = ycol[c];
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < (size_t)m * m; g += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(g / m), i = (int)(g % m);
    const double s = fd_s(i, n) * fd_s(j, n);
    const int nsides = (i == 0 || i == n) + (j == 0 || j == n);
    const double2 x0 = x[g];
    // centre (4 - k^2 h^2 - 2 i k h nsides)
    double re = (4.0 - kh2) * x0.x + 2.0 * kh * nsides * x0.y;
    double im = (4.0 - kh2) * x0.y - 2.0 * kh * nsides * x0.x;
    // four neighbours; a missing one is the ghost, i.e. the mirror node
    const size_t e_ = (i < n) ? g + 1 : g - 1, w_ = (i > 0) ? g - 1 : g + 1;
    const size_t n_ = (j < n) ? g + m : g - m, s_ = (j > 0) ? g - m : g + m;
    re -= x[e_].x + x[w_].x + x[n_].x + x[s_].x;
    im -= x[e_].y + x[w_].y + x[n_].y + x[s_].y;
    y[g] = make_double2(s * re, s * im);
  }
}

// b = s (-h^2 f) with f a sum of Gaussians (rows x0, y0, sigma, re, im)
__global__ void fd_load_kernel(const double* __restrict__ src, int nsrc, int n, double2* __restrict__ b) {
  const int m = n + 1;
  const double h = 1.0 / n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < (size_t)m * m; g += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(g / m), i = (int)(g % m);
    const double x = i * h, yv = j * h;
    double2 acc = make_double2(0, 0);
    for (int q = 0; q < nsrc; ++q) {
      const double* p = src + 5 * q;
      const double dx = x - p[0], dy = yv - p[1];
      const double e = exp(-(dx * dx + dy * dy) / (2.0 * p[2] * p[2]));
      acc.x += p[3] * e;
      acc.y += p[4] * e;
    }
    const double w = -h * h * fd_s(i, n) * fd_s(j, n);
    b[g] = make_double2(w * acc.x, w * acc.y);
  }
}

// ------------------------------------------------------------------ host side
// columns per sweep pass: the step kernel stages one input line of m x C complex values as
// three FP64 planes in shared memory (at most 192 KB)
static int fd_chunk(int m) { return std::max(1, std::min(32, (int)(192 * 1024 / ((size_t)m * 3 * sizeof(double))))); }

int fd_setup(Engine& E) {
  FdState* st = new (std::nothrow) FdState();
  if (!st) return HH_ENOMEM;
  E.fd = st;
  const int n = E.n, N = E.N, R = E.R, m = E.m;
  st->a.resize(N);
  st->L.resize(N);
  for (int s = 0; s < N; ++s) {
    const int a = std::max(0, s * R - 1), b = std::min(n, (s + 1) * R + 1);
    st->a[s] = a;
    st->L[s] = b - a + 1;
    st->Lmax = std::max(st->Lmax, st->L[s]);
  }
  st->nchain = st->Lmax - 1;
  std::vector<int>& tops = st->tops;
  for (int s = 0; s < N; ++s)
    if (std::find(tops.begin(), tops.end(), st->L[s]) == tops.end()) tops.push_back(st->L[s]);
  st->nblk = st->nchain + (int)tops.size();
  const size_t blk = (size_t)m * E.ldf;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  if ((size_t)(st->nblk + 3) * blk * sizeof(double2) + (64ull << 20) > free_b)
    return (set_error("five-point strip inverses do not fit in free device memory"), HH_ENOMEM);
  double2 *Dbnd = nullptr, *Dint = nullptr;
  if (E.dmalloc((void**)&st->F, st->nblk * blk * sizeof(double2)) || E.dmalloc((void**)&Dbnd, blk * sizeof(double2)) ||
      E.dmalloc((void**)&Dint, blk * sizeof(double2))) {
    E.dfree(Dbnd);
    return HH_ENOMEM;
  }
  cudaMemsetAsync(Dbnd, 0, blk * sizeof(double2), E.stream);
  cudaMemsetAsync(Dint, 0, blk * sizeof(double2), E.stream);
  fd_line_block_kernel<<<E.grid_for((size_t)m * m), 256, 0, E.stream>>>(Dbnd, n, E.ldf, E.k, 1);
  fd_line_block_kernel<<<E.grid_for((size_t)m * m), 256, 0, E.stream>>>(Dint, n, E.ldf, E.k, 0);
  E.count_launch(2);
  std::vector<double2*> out(st->nblk);
  for (int q = 0; q < st->nblk; ++q) out[q] = st->F + (size_t)q * blk;
  auto form = [&](int q, double2* S) -> int {
    if (q == 0) {
      fd_schur_kernel<<<E.grid_for((size_t)m * m), 256, 0, E.stream>>>(Dbnd, nullptr, S, n, E.ldf);
    } else if (q < st->nchain) {
      fd_schur_kernel<<<E.grid_for((size_t)m * m), 256, 0, E.stream>>>(Dint, out[q - 1], S, n, E.ldf);
    } else {
      const int L = tops[q - st->nchain];
      fd_schur_kernel<<<E.grid_for((size_t)m * m), 256, 0, E.stream>>>(Dbnd, out[L - 2], S, n, E.ldf);
    }
    E.count_launch();
    return cudaGetLastError() == cudaSuccess ? HH_OK : HH_ECUDA;
  };
  const int rc = invert_chain_fp64(E, st->nblk, form, out.data());
  cudaStreamSynchronize(E.stream);
  E.dfree(Dbnd);
  E.dfree(Dint);
  if (rc) return rc;
  cudaFuncSetAttribute((const void*)fd_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fd_step_smem(m, fd_chunk(m)));
  return E.check_device_error("five-point setup");
}

void fd_free(Engine& E) {
  FdState* st = E.fd;
  if (!st) return;
  E.dfree(st->F); E.dfree(st->X); E.dfree(st->Y); E.dfree(st->sub); E.dfree(st->fbuf);
  delete st;
  E.fd = nullptr;
}

static int fd_ensure(Engine& E, int C) {
  FdState* st = E.fd;
  if (C <= st->Cmax) return HH_OK;
  E.dfree(st->X); E.dfree(st->Y); E.dfree(st->sub); E.dfree(st->fbuf);
  st->X = st->Y = st->sub = st->fbuf = nullptr;
  st->Cmax = 0;
  const size_t line = (size_t)E.m * C;
  if (E.dmalloc((void**)&st->X, line * E.m * sizeof(double2)) || E.dmalloc((void**)&st->Y, line * E.m * sizeof(double2)) ||
      E.dmalloc((void**)&st->sub, line * st->Lmax * E.N * sizeof(double2)) ||
      E.dmalloc((void**)&st->fbuf, line * st->Lmax * sizeof(double2)))
    return HH_ENOMEM;
  st->Cmax = C;
  return HH_OK;
}

int fd_reserve(Engine& E, int C) { return fd_ensure(E, std::min(C, fd_chunk(E.m))); }
int fd_blocks(const Engine& E) { return E.fd ? E.fd->nblk : 0; }

// inverse for line l of a subdomain with L lines
static const double2* fd_block(const FdState* st, const Engine& E, int l, int L) {
  const size_t blk = (size_t)E.m * E.ldf;
  if (l < L - 1) return st->F + (size_t)l * blk;
  const int q = (int)(std::find(st->tops.begin(), st->tops.end(), L) - st->tops.begin());
  return st->F + (size_t)(st->nchain + q) * blk;
}

static void fd_step(Engine& E, const double2* F, const double2* a, const double2* b, const double2* base, double2* out,
                    int C) {
  const int grid = (E.m + FD_ROWS - 1) / FD_ROWS;
  fd_step_kernel<<<grid, 32 * FD_ROWS, fd_step_smem(E.m, C), E.stream>>>(F, E.ldf, a, b, base, out, E.n, C);
  E.count_launch();
}

// block Thomas on subdomain s (its right-hand side in fbuf), solution into sub[s]
static void fd_thomas(Engine& E, int s, int C) {
  FdState* st = E.fd;
  const size_t line = (size_t)E.m * C;
  const int L = st->L[s];
  double2* u = st->sub + (size_t)s * st->Lmax * line;
  for (int l = 0; l < L; ++l)
    fd_step(E, fd_block(st, E, l, L), st->fbuf + l * line, l ? u + (l - 1) * line : nullptr, nullptr, u + l * line, C);
  for (int l = L - 2; l >= 0; --l)
    fd_step(E, fd_block(st, E, l, L), nullptr, u + (l + 1) * line, u + l * line, u + l * line, C);
}

static void fd_rhs(Engine& E, int s, int C, int lo_s, int hi_s) {
  FdState* st = E.fd;
  const size_t line = (size_t)E.m * C;
  const double2* lo = lo_s >= 0 ? st->sub + (size_t)lo_s * st->Lmax * line : nullptr;
  const double2* hi = hi_s >= 0 ? st->sub + (size_t)hi_s * st->Lmax * line : nullptr;
  fd_rhs_kernel<<<E.grid_for((size_t)st->L[s] * line), 256, 0, E.stream>>>(
      st->X, st->fbuf, st->a[s], st->L[s], lo, lo_s >= 0 ? st->a[lo_s] : 0, hi, hi_s >= 0 ? st->a[hi_s] : 0, E.n, C,
      E.k);
  E.count_launch();
}

static void fd_place(Engine& E, int s, int C) {
  FdState* st = E.fd;
  const size_t line = (size_t)E.m * C;
  fd_place_kernel<<<E.grid_for((size_t)st->L[s] * line), 256, 0, E.stream>>>(st->sub + (size_t)s * st->Lmax * line,
                                                                            st->Y, st->a[s], st->L[s], E.n, C);
  E.count_launch();
}

// M_d^{-1} for C columns: column c = scale[c] src[c] in direction codes[(c0 + c) % t] (c0: the
// first column's index in the caller's tables), written to dst[c].  Double sweeps (Eqs. (2),
// (3)) or forward sweeps only; columns in passes of fd_chunk(m).
int fd_precondition(Engine& E, const double2* const* src, const double* scale, int C, int t, int4 codes,
                    double2* const* dst, bool single) {
  FdState* st = E.fd;
  const int Cc = std::min(C, fd_chunk(E.m));
  if (fd_ensure(E, Cc)) return HH_ENOMEM;
  const int N = E.N;
  for (int c0 = 0; c0 < C; c0 += Cc) {
    const int cc = std::min(Cc, C - c0);
    // the direction of column c0 + c is codes[(c0 + c) % t]: rotate the codes to start at c0
    int cd[4] = {codes.x, codes.y, codes.z, codes.w};
    int rot[4];
    for (int d = 0; d < 4; ++d) rot[d] = cd[(c0 + d) % t];
    const int4 rc4 = make_int4(rot[0], rot[1], rot[2], rot[3]);
    const size_t total = (size_t)E.m * E.m * cc;
    fd_pack_kernel<<<E.grid_for(total), 256, 0, E.stream>>>(src + c0, scale ? scale + c0 : nullptr, cc, t, rc4, st->X,
                                                            E.n);
    E.count_launch();
    for (int s = 0; s < N; ++s) {
      fd_rhs(E, s, cc, s > 0 ? s - 1 : -1, -1);
      fd_thomas(E, s, cc);
    }
    if (single) {
      for (int s = 0; s < N; ++s) fd_place(E, s, cc);  // overlaps keep the higher subdomain's values
    } else {
      for (int s = N - 2; s >= 0; --s) {
        fd_rhs(E, s, cc, s > 0 ? s - 1 : -1, s + 1);
        fd_thomas(E, s, cc);
      }
      for (int s = N - 1; s >= 0; --s) fd_place(E, s, cc);  // overlaps keep the lower subdomain's values
    }
    fd_unpack_kernel<<<E.grid_for(total), 256, 0, E.stream>>>(st->Y, dst + c0, cc, t, rc4, E.n);
    E.count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? HH_OK : HH_ECUDA;
}

void fd_operator(Engine& E, const double2* const* xcol, double2* const* ycol, int ncols) {
  const size_t D = (size_t)E.m * E.m;
  fd_operator_kernel<<<dim3(std::max(1u, E.grid_for(D * ncols) / ncols), ncols), 256, 0, E.stream>>>(xcol, ycol, ncols,
                                                                                                   E.n, E.k);
  E.count_launch();
}

void fd_load(Engine& E, const double* dsrc, int nsrc, double2* b) {
  fd_load_kernel<<<E.grid_for((size_t)E.m * E.m), 256, 0, E.stream>>>(dsrc, nsrc, E.n, b);
  E.count_launch();
}

}  // namespace hh
