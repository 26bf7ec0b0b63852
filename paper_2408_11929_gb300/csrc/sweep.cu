// Batched directional double sweeps (Section 2, Eqs. (2)-(3)) as one persistent launch.
//
// Frame.  The mesh (cells cut along SW-NE diagonals) is invariant under the transpose
// (i, j) -> (j, i) and the half-turn (i, j) -> (n-i, n-j), and so is A.  The four sweeps
// are images of the bottom-to-top sweep BT under these maps (LR = transpose, TB = half
// turn, RL = both, each with its strips mapped alike, the last strip visited owning the
// extra line).  Every preconditioner application is therefore a BT sweep of a permuted
// copy of its input: the pack kernel writes each (right-hand side, direction) pair as one
// column of a line-major array X[line][node][column], one persistent kernel sweeps all
// columns together -- every factor block read once per step serves all directions and
// right-hand sides -- and the unpack kernel maps the columns back.
//
// Sweep in the BT frame, strips s = 0..N-1 of lines [sR, sR+R-1] (last: R+1 lines), with
// the block Thomas factors F_j = S_j^{-1} of the strip matrix (setup.cu):
//   forward  (strip s, j = 0..len-1): y_j = F_j (r_j - L y_{j-1})  (y_{-1}: last line of strip s-1)
//            then x_j = y_j - F_j U x_{j+1} for j = len-2..0     (v_s = x)
//   backward (strip s = N-2..0): z_{R-1} = F_{R-1} U u_{s+1}(first line),
//            z_j = F_j (-U z_{j+1}), u_j = v_j - z_j            (u_{N-1} = v_{N-1}, Section 2)
// L couples a line to the one below (vertical edge, cell diagonal), U = L^T to the one above.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "engine.h"

namespace hh {

std::vector<SweepOp> build_schedule(int n, int N, bool double_sweep) {
  std::vector<SweepOp> ops;
  const int R = n / N;
  auto mk_op = [](int f, int out_line, int out_sub, int zsave, int base, int cpl, int src, int cline, int neg) {
    SweepOp o{};
    o.f = f; o.out_line = out_line; o.out_sub = out_sub; o.zsave = zsave; o.base_line = base;
    o.cpl = cpl; o.cpl_src = src; o.cpl_line = cline; o.cpl_neg = neg;
    return o;
  };
  for (int s = 0; s < N; ++s) {
    const int a = s * R, len = (s == N - 1) ? R + 1 : R;
    for (int j = 0; j < len; ++j) {
      const int l = a + j;
      ops.push_back(mk_op(j, l, 0, -1, l, l > 0 ? 1 : 0, 0, l - 1, 1));
    }
    for (int j = len - 2; j >= 0; --j) {
      const int l = a + j;
      ops.push_back(mk_op(j, l, 1, -1, -1, 2, 0, l + 1, 0));
    }
  }
  if (double_sweep) {
    for (int s = N - 2; s >= 0; --s) {
      const int a = s * R, b = a + R - 1;
      ops.push_back(mk_op(R - 1, b, 1, 0, -1, 2, 0, b + 1, 0));
      int slot = 0;
      for (int j = R - 2; j >= 0; --j) {
        ops.push_back(mk_op(j, a + j, 1, 1 - slot, -1, 2, 1 + slot, 0, 1));
        slot = 1 - slot;
      }
    }
  }
  return ops;
}

// BT-frame node (i, l) of a column with direction code c -> grid node (io, jo)
__device__ __forceinline__ void frame_map(int code, int i, int l, int n, int& io, int& jo) {
  switch (code) {
    case DC_BT: io = i; jo = l; break;
    case DC_TB: io = n - i; jo = n - l; break;
    case DC_LR: io = l; jo = i; break;
    default: io = n - l; jo = n - i; break;  // DC_RL
  }
}

__device__ __forceinline__ int code_of(int4 codes, int d) {
  return d == 0 ? codes.x : (d == 1 ? codes.y : (d == 2 ? codes.z : codes.w));
}

template <typename R>
__global__ void pack_kernel(const double2* const* __restrict__ srcptr, const double* __restrict__ scale, int C,
                            int t, int4 codes, int n, typename Cx<R>::T* __restrict__ X) {
  using T = typename Cx<R>::T;
  const int m = n + 1;
  const size_t total = (size_t)m * m * C;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % C);
    const size_t node = idx / C;
    const int l = (int)(node / m), i = (int)(node % m);
    int io, jo;
    frame_map(code_of(codes, c % t), i, l, n, io, jo);
    const double2 v = srcptr[c][(size_t)jo * m + io];
    const double s = scale[c];
    X[idx] = mk<T>(v.x * s, v.y * s);
  }
}

template <typename R>
__global__ void unpack_kernel(const typename Cx<R>::T* __restrict__ X, int C, int t, int4 codes, int n,
                              double2* __restrict__ dst, size_t stride) {
  const int m = n + 1;
  const size_t total = (size_t)m * m * C;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % C);
    const size_t node = idx / C;
    const int l = (int)(node / m), i = (int)(node % m);
    int io, jo;
    frame_map(code_of(codes, c % t), i, l, n, io, jo);
    dst[(size_t)c * stride + (size_t)jo * m + io] = to_d(X[idx]);
  }
}

// Persistent sweep.  CTA b owns rows [b*rp, min(m, (b+1)*rp)) of every block step.  Each
// step: every CTA builds the full input line x (m x CT columns, in shared memory) from
// Rin and the coupled line, multiplies its rows of F_f by it (one warp per row and column
// group, warp-shuffle reduction), writes its rows of the output, then all CTAs meet at a
// bounded grid barrier.  Columns are processed in tiles of CT that fit shared memory.
template <typename R, int CC>
__global__ void __launch_bounds__(256) sweep_kernel(const typename Cx<R>::T* __restrict__ F, int ldf, int m,
                                                    int C, int CT, const typename Cx<R>::T* __restrict__ Rin,
                                                    typename Cx<R>::T* V, typename Cx<R>::T* Zt,
                                                    const SweepOp* __restrict__ ops, int nops, Coef cf,
                                                    unsigned* bar, int* err, long long budget) {
  using T = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* vert_s = reinterpret_cast<T*>(smem_raw);
  T* x_s = vert_s + ((m + 1) & ~1);
  const int rp = (m + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * rp;
  const int r1 = min(m, r0 + rp);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const size_t lineC = (size_t)m * C;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double2 v = cf.vert(i);
    vert_s[i] = mk<T>(v.x, v.y);
  }
  const R dg = (R)cf.diag();
  unsigned target = 0;
  __syncthreads();
  for (int op = 0; op < nops; ++op) {
    const SweepOp o = ops[op];
    const T* src = (o.cpl_src == 0) ? V + (size_t)o.cpl_line * lineC : Zt + (size_t)(o.cpl_src - 1) * lineC;
    const T* base = o.base_line >= 0 ? Rin + (size_t)o.base_line * lineC : nullptr;
    const T* Fb = F + (size_t)o.f * m * ldf;
    T* out = V + (size_t)o.out_line * lineC;
    T* zs = o.zsave >= 0 ? Zt + (size_t)o.zsave * lineC : nullptr;
    for (int c0 = 0; c0 < C; c0 += CT) {
      const int ct = min(CT, C - c0);
      for (int idx = threadIdx.x; idx < m * ct; idx += blockDim.x) {
        const int i = idx / ct, cc = idx - i * ct;
        const size_t g = (size_t)i * C + c0 + cc;
        T v = base ? __ldg(base + g) : mk<T>(0, 0);
        if (o.cpl) {
          T cp = cmul(vert_s[i], __ldcg(src + g));
          if (o.cpl == 1 && i >= 1) { const T y = __ldcg(src + g - C); cp.x += dg * y.x; cp.y += dg * y.y; }
          if (o.cpl == 2 && i + 1 < m) { const T y = __ldcg(src + g + C); cp.x += dg * y.x; cp.y += dg * y.y; }
          v = o.cpl_neg ? csub(v, cp) : cadd(v, cp);
        }
        x_s[idx] = v;
      }
      __syncthreads();
      const int ngrp = ct / CC;
      const int nwork = (r1 > r0 ? r1 - r0 : 0) * ngrp;
      for (int w = wid; w < nwork; w += nw) {
        const int row = r0 + w / ngrp, cg = (w % ngrp) * CC;
        T acc[CC];
#pragma unroll
        for (int q = 0; q < CC; ++q) acc[q] = mk<T>(0, 0);
        const T* Fr = Fb + (size_t)row * ldf;
        for (int i = lane; i < m; i += 32) {
          const T fv = __ldg(Fr + i);
          const T* xr = x_s + i * ct + cg;
#pragma unroll
          for (int q = 0; q < CC; ++q) cfma(acc[q], fv, xr[q]);
        }
#pragma unroll
        for (int q = 0; q < CC; ++q)
#pragma unroll
          for (int s = 16; s; s >>= 1) acc[q] = cadd(acc[q], shfl_xor(acc[q], s));
        if (lane < CC) {
          T z = acc[0];
#pragma unroll
          for (int q = 1; q < CC; ++q)
            if (lane == q) z = acc[q];
          const size_t g = (size_t)row * C + c0 + cg + lane;
          if (o.out_sub) out[g] = csub(__ldcg(out + g), z);
          else out[g] = z;
          if (zs) zs[g] = z;
        }
      }
      __syncthreads();
    }
    if (op + 1 < nops) {
      if (!grid_sync(bar, target, err, budget)) return;
    }
  }
}

int Engine::ensure_sweep_ws(int C) {
  if ((size_t)C <= w_cap_cols) return HH_OK;
  dfree(w_rin); dfree(w_v); dfree(w_zt);
  w_rin = w_v = w_zt = nullptr;
  w_cap_cols = 0;
  const size_t line = (size_t)m * C * sweep_elem();
  if (dmalloc(&w_rin, line * m) || dmalloc(&w_v, line * m) || dmalloc(&w_zt, line * 2)) return HH_ENOMEM;
  w_cap_cols = C;
  return HH_OK;
}

template <typename R, int CC>
static cudaError_t launch_sweep_t(Engine& E, const void* Rin, void* V, void* Zt, int C, bool single) {
  using T = typename Cx<R>::T;
  const int m = E.m;
  const int grid = std::min(E.num_sms, m);
  const size_t cap = 200 * 1024;
  const size_t vert_bytes = (size_t)((m + 1) & ~1) * sizeof(T);
  int CT = (int)((cap - vert_bytes) / ((size_t)m * sizeof(T)));
  CT = std::min(CT, C);
  CT = (CT / CC) * CC;
  if (CT < CC) CT = CC;
  const size_t smem = vert_bytes + (size_t)m * CT * sizeof(T);
  auto fn = sweep_kernel<R, CC>;
  cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const T* Fp = reinterpret_cast<const T*>(E.factors);
  const T* Rp = reinterpret_cast<const T*>(Rin);
  T* Vp = reinterpret_cast<T*>(V);
  T* Zp = reinterpret_cast<T*>(Zt);
  const SweepOp* ops = single ? E.d_ops_single : E.d_ops;
  int nops = single ? E.nops_single : E.nops_double;
  int ldf = E.ldf;
  long long budget = E.opts.timeout_cycles;
  void* args[] = {(void*)&Fp, (void*)&ldf, (void*)&E.m, (void*)&C, (void*)&CT, (void*)&Rp, (void*)&Vp, (void*)&Zp,
                  (void*)&ops, (void*)&nops, (void*)&E.coef, (void*)&E.bar, (void*)&E.err, (void*)&budget};
  cudaMemsetAsync(E.bar, 0, sizeof(unsigned), E.stream);
  return E.launch_coop((const void*)fn, grid, 256, smem, args);
}

int Engine::run_sweep(const void* Rin, void* V, void* Zt, int C, bool single) {
  const int nops = single ? nops_single : nops_double;
  const double elem = (double)sweep_elem();
  const double fbytes = (double)nops * m * m * elem + 2.0 * m * m * C * elem;
  tick_begin(K_SWEEP);
  cudaError_t ce;
  int cc = (C % 4 == 0) ? 4 : ((C % 2 == 0) ? 2 : 1);
  // the shared-memory input tile must hold at least one column group
  while (cc > 1 && (size_t)m * cc * sweep_elem() > 190 * 1024) cc >>= 1;
  if (precision == HH_PREC_FP32) {
    ce = cc == 4 ? launch_sweep_t<float, 4>(*this, Rin, V, Zt, C, single)
                 : (cc == 2 ? launch_sweep_t<float, 2>(*this, Rin, V, Zt, C, single)
                            : launch_sweep_t<float, 1>(*this, Rin, V, Zt, C, single));
  } else {
    ce = cc == 4 ? launch_sweep_t<double, 4>(*this, Rin, V, Zt, C, single)
                 : (cc == 2 ? launch_sweep_t<double, 2>(*this, Rin, V, Zt, C, single)
                            : launch_sweep_t<double, 1>(*this, Rin, V, Zt, C, single));
  }
  tick_end(K_SWEEP, fbytes, (double)nops * m * m * C * 8.0);
  last_columns = C;
  if (ce != cudaSuccess) { set_cuda_error(ce, "sweep launch"); return HH_ECUDA; }
  return HH_OK;
}

// launch helpers used by krylov.cu / api.cu
template <typename R>
static void launch_pack_t(Engine& E, const double2* const* srcptr, const double* scale, int C, int t, int4 codes,
                          void* X) {
  pack_kernel<R><<<E.grid_for((size_t)E.m * E.m * C), 256, 0, E.stream>>>(srcptr, scale, C, t, codes, E.n,
                                                                           reinterpret_cast<typename Cx<R>::T*>(X));
  E.count_launch();
}
template <typename R>
static void launch_unpack_t(Engine& E, const void* X, int C, int t, int4 codes, double2* dst, size_t stride) {
  unpack_kernel<R><<<E.grid_for((size_t)E.m * E.m * C), 256, 0, E.stream>>>(
      reinterpret_cast<const typename Cx<R>::T*>(X), C, t, codes, E.n, dst, stride);
  E.count_launch();
}

void launch_pack(Engine& E, const double2* const* srcptr, const double* scale, int C, int t, int4 codes, void* X) {
  if (E.precision == HH_PREC_FP32) launch_pack_t<float>(E, srcptr, scale, C, t, codes, X);
  else launch_pack_t<double>(E, srcptr, scale, C, t, codes, X);
}
void launch_unpack(Engine& E, const void* X, int C, int t, int4 codes, double2* dst, size_t stride) {
  if (E.precision == HH_PREC_FP32) launch_unpack_t<float>(E, X, C, t, codes, dst, stride);
  else launch_unpack_t<double>(E, X, C, t, codes, dst, stride);
}

}  // namespace hh
