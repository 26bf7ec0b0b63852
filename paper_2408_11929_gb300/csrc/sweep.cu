// Batched directional double sweeps (Section 2, Eqs. (2)-(3)).
//
// Frame.  The mesh (cells cut along SW-NE diagonals) is invariant under the transpose
// (i, j) -> (j, i) and the half-turn (i, j) -> (n-i, n-j), and so is A.  The four sweeps
// are images of the bottom-to-top sweep BT under these maps (LR = transpose, TB = half
// turn, RL = both, each with its strips mapped alike, the last strip visited owning the
// extra line).  Every preconditioner application is therefore a BT sweep of a permuted copy
// of its input: the pack kernel writes each (right-hand side, direction) pair as one column
// and all columns are swept together -- every strip factor read serves all directions,
// right-hand sides and strips -- and the unpack kernel maps the columns back.
//
// Strip-interleaved layout.  Strip s (s = 0..N-1) owns BT-frame lines s R + j, j = 0..R-1
// (the last strip also j = R).  Sweep arrays are X[j][i][s][c]: line-in-strip j, node i,
// strip s, column c, so that one step of a block-Thomas recurrence over all strips is one
// GEMM  F_j (m x m) * X[j] (m x N C).
//
// The double sweep (block Gauss-Seidel forward then backward over the strips) is computed
// exactly, reorganised so that only the interface values travel from strip to strip:
//   F1  w_s = D^{-1} r_s for every strip at once (block Thomas, 2R+1 GEMM steps);
//   F2  interface chain t_s = w_s[R-1] - G t_{s-1},  G = D^{-1}[R-1, 0] L       (N-2 steps),
//       where t_s is the last line of the forward solution v_s;
//   F3  v_s = w_s + D^{-1} e_0 (-L t_{s-1}) for s >= 1 (block Thomas with a right-hand side
//       on the first line only, 2R+1 GEMM steps; the last lines already hold t_s);
//   B1  interface chain of the backward sweep on the first lines:
//       u_s[0] = v_s[0] - K u_{s+1}[0],  K = D^{-1}[0, R-1] U = (D^{-1}[R-1, 0])^T U  (N-1 steps;
//       D is complex symmetric, so D^{-1}[0, R-1] is the transpose of D^{-1}[R-1, 0]);
//   B2  u_s[j] = v_s[j] - (D^{-1} e_{R-1} U u_{s+1}[0])[j] for j = R-1..1 (R-1 GEMM steps);
//       u_{N-1} = v_{N-1} (one solve in the last strip, Section 2).
// F_j are the block-Thomas inverses of the strip matrix, G and K come from setup.cu.
// A single (forward-only) sweep stops after F3.
#include <algorithm>
#include <cstdio>
#include <vector>

#include <cudaTypedefs.h>
#include <cstring>
#include <string>
#include <type_traits>

#include "common.cuh"
#include "engine.h"
#include "gemm.cuh"
#include "tc_gemm.cuh"

namespace hh {

std::vector<SweepStep> build_steps(int n, int N, bool double_sweep) {
  std::vector<SweepStep> st;
  const int R = n / N, last = N - 1;
  const int FG = R + 1, FK = R + 2;  // block indices of G and K
  auto mk_step = [](int f, int s0, int ns) {
    SweepStep x{};
    x.f = f; x.s0 = s0; x.ns = ns;
    x.base = SB_NONE; x.src = SB_NONE; x.cpl = XC_NONE; x.acc = SB_NONE;
    return x;
  };
  // F1: forward elimination, all strips (line R only in the last strip)
  for (int j = 0; j <= R; ++j) {
    SweepStep x = mk_step(j, j == R ? last : 0, j == R ? 1 : N);
    x.base = SB_RIN; x.base_j = j;
    if (j >= 1) { x.src = SB_V; x.src_j = j - 1; x.cpl = XC_LOWER; x.neg = 1; }
    x.out = SB_V; x.out_j = j; x.out_mode = OUT_SET;
    st.push_back(x);
  }
  // F1: back substitution (line R-1 has a successor only in the last strip)
  for (int j = R - 1; j >= 0; --j) {
    SweepStep x = mk_step(j, j == R - 1 ? last : 0, j == R - 1 ? 1 : N);
    x.src = SB_V; x.src_j = j + 1; x.cpl = XC_UPPER;
    x.out = SB_V; x.out_j = j; x.out_mode = OUT_SUB;
    st.push_back(x);
  }
  if (N >= 2) {
    // F2: interface chain on the last lines
    for (int s = 1; s <= N - 2; ++s) {
      SweepStep x = mk_step(FG, s, 1);
      x.src = SB_V; x.src_j = R - 1; x.src_ds = -1; x.cpl = XC_IDENT;
      x.out = SB_V; x.out_j = R - 1; x.out_mode = OUT_SUB;
      st.push_back(x);
    }
    // F3: responses to the first-line coupling -L t_{s-1}, strips 1..N-1 (corrections in W)
    for (int j = 0; j <= R; ++j) {
      SweepStep x = mk_step(j, j == R ? last : 1, j == R ? 1 : N - 1);
      x.src = (j == 0) ? SB_V : SB_W;
      x.src_j = (j == 0) ? R - 1 : j - 1;
      x.src_ds = (j == 0) ? -1 : 0;
      x.cpl = XC_LOWER; x.neg = 1;
      x.out = SB_W; x.out_j = j; x.out_mode = OUT_SET;
      if (j == R) { x.acc = SB_V; x.acc_j = R; x.acc_mode = OUT_ADD; }
      st.push_back(x);
    }
    for (int j = R - 1; j >= 0; --j) {
      SweepStep x = mk_step(j, j == R - 1 ? last : 1, j == R - 1 ? 1 : N - 1);
      x.src = SB_W; x.src_j = j + 1; x.cpl = XC_UPPER;
      x.out = SB_W; x.out_j = j; x.out_mode = OUT_SUB;
      x.acc = SB_V; x.acc_j = j; x.acc_mode = OUT_ADD;
      st.push_back(x);
    }
  }
  if (double_sweep && N >= 2) {
    // B1: interface chain on the first lines, last strip first
    for (int s = N - 2; s >= 0; --s) {
      SweepStep x = mk_step(FK, s, 1);
      x.src = SB_V; x.src_j = 0; x.src_ds = 1; x.cpl = XC_IDENT;
      x.out = SB_V; x.out_j = 0; x.out_mode = OUT_SUB;
      st.push_back(x);
    }
    // B2: responses to the last-line coupling U u_{s+1}[0], lines R-1..1 of strips 0..N-2
    for (int j = R - 1; j >= 1; --j) {
      SweepStep x = mk_step(j, 0, N - 1);
      if (j == R - 1) { x.src = SB_V; x.src_j = 0; x.src_ds = 1; x.cpl = XC_UPPER; x.neg = 0; }
      else { x.src = SB_W; x.src_j = j + 1; x.cpl = XC_UPPER; x.neg = 1; }
      x.out = SB_W; x.out_j = j; x.out_mode = OUT_SET;
      x.acc = SB_V; x.acc_j = j; x.acc_mode = OUT_SUB;
      st.push_back(x);
    }
  }
  return st;
}

static int ceil_log2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

int max_bcr_depth(int R) {
  int d = 0;
  while (d < 7 && R % (2 << d) == 0) ++d;
  return d;
}

bool twisted_possible(int R, int N, int form) { return form != 0 && N >= 2 && R >= 4; }

BlockDir block_directory(int R, int N, int form, unsigned depths, bool twisted) {
  BlockDir bd;
  bd.total = R + 3;
  if (form != 0 && N >= 2) {
    bd.LF = N >= 3 ? ceil_log2(N - 1) : 0;
    bd.LB = ceil_log2(N);
    bd.iY = R + 3;
    bd.iYL = bd.iY + R;
    bd.iZ = bd.iYL + R + 1;
    bd.iGp = bd.iZ + (R - 1);
    bd.iKp = bd.iGp + std::max(0, bd.LF - 1);
    bd.total = bd.iKp + std::max(0, bd.LB - 1);
  }
  const int dlim = max_bcr_depth(R);
  for (int d = 1; d <= dlim; ++d)
    if (depths & (1u << d)) bd.dmax = d;
  if (bd.dmax > 0) {
    bd.iLev = bd.total;
    bd.total += 5 * bd.dmax;
    for (int d = 1; d <= bd.dmax; ++d)
      if (depths & (1u << d)) {
        bd.iDeep[d] = bd.total;
        bd.total += 3 * (R >> d) + 1;
      }
  }
  if (twisted && twisted_possible(R, N, form)) {
    bd.twq = R / 2;
    bd.iTw = bd.total;
    bd.iTwM = bd.iTw + (R - 1 - bd.twq);
    bd.iZ0 = bd.iTwM + 1;
    bd.total = bd.iZ0 + 1;
  }
  return bd;
}

// F1 (w_s = D^{-1} r_s for every strip) by block cyclic reduction of depth d >= 1 (Section 2's
// strip solve is block LU of a block-tridiagonal matrix; odd-even reduction orders it so
// that every level is one grouped step over all its lines and strips):
//   forward, level l = 1..d (h = 2^(l-1), source Rin at l = 1, else W): the kept lines
//     p = 0, 2h, 4h, .. (and R in the last strip) get
//     r^l_p = r^(l-1)_p - (L Dinv) r^(l-1)_{p-h} - (U Dinv) r^(l-1)_{p+h}   (into W);
//   the reduced system (lines p = i 2^d) by block Thomas with dense couplings:
//     y_i = F_i r_i for every line at once, then y_i -= G_i y_{i-1} (chain), the last strip's
//     top line y_top -= G_top y_{nd-1}, then u_i = y_i - H_i u_{i+1} (chain; the strips before
//     the last start one line lower: their top line has nothing above it);
//   back substitution, level l = d..1: the eliminated lines p = h, 3h, .. get
//     u_p = Dinv r^(l-1)_p - (Dinv L) u_{p-h} - (Dinv U) u_{p+h}   (into V),
//   the top eliminated line of the strips before the last without the last term.
static void append_bcr_f1(std::vector<SweepPhase>& prog, int R, int N, int d, const BlockDir& bd) {
  auto term = [](int f, int arr, int line, int neg) { return GTerm{f, arr, line, 0, neg, 0, 0, 0}; };
  auto task = [](std::initializer_list<GTerm> terms, int out_arr, int out_line, int base_arr, int base_line,
                 int mode, int s0, int ns) {
    GTask t{};
    t.nterm = 0;
    for (const GTerm& g : terms) t.term[t.nterm++] = g;
    t.out_arr = out_arr; t.out_line = out_line;
    t.base_arr = base_arr; t.base_line = base_line;
    t.mode = mode; t.s0 = s0; t.ns = ns;
    return t;
  };
  auto group = [](std::vector<GTask> ts) {
    SweepPhase p;
    p.kind = PH_GROUP;
    for (const GTask& t : ts)
      if (t.ns > 0) p.tasks.push_back(t);
    return p;
  };
  const int last = N - 1, nl = N - 1;  // the last strip; the strips before it
  for (int l = 1; l <= d; ++l) {
    const int h = 1 << (l - 1), src = l == 1 ? SB_RIN : SB_W;
    const int lev = bd.iLev + 5 * (l - 1), AF = lev + 1, BF = lev + 2;
    std::vector<GTask> ts;
    ts.push_back(task({term(BF, src, h, 1)}, SB_W, 0, src, 0, OUT_SET, 0, N));
    for (int p = 2 * h; p < R; p += 2 * h)
      ts.push_back(task({term(AF, src, p - h, 1), term(BF, src, p + h, 1)}, SB_W, p, src, p, OUT_SET, 0, N));
    ts.push_back(task({term(AF, src, R - h, 1)}, SB_W, R, src, R, OUT_SET, last, 1));
    prog.push_back(group(ts));
  }
  const int nd = R >> d, S = 1 << d, b = bd.iDeep[d];
  const int iF = b, iFtop = b + nd, iGtop = b + 2 * nd, iH = b + 2 * nd + 1;
  auto iG = [&](int i) { return b + nd + i; };
  {
    std::vector<GTask> ts;
    for (int i = 0; i < nd; ++i) ts.push_back(task({term(iF + i, SB_W, i * S, 0)}, SB_V, i * S, SB_NONE, 0, OUT_SET, 0, N));
    ts.push_back(task({term(iFtop, SB_W, R, 0)}, SB_V, R, SB_NONE, 0, OUT_SET, last, 1));
    prog.push_back(group(ts));
  }
  for (int i = 1; i < nd; ++i)
    prog.push_back(group({task({term(iG(i), SB_V, (i - 1) * S, 1)}, SB_V, i * S, SB_NONE, 0, OUT_ADD, 0, N)}));
  prog.push_back(group({task({term(iGtop, SB_V, R - S, 1)}, SB_V, R, SB_NONE, 0, OUT_ADD, last, 1)}));
  for (int q = 0; q < nd; ++q) {
    std::vector<GTask> ts;
    const int il = nd - 1 - q;  // the last strip's line
    ts.push_back(task({term(iH + il, SB_V, (il + 1) * S, 1)}, SB_V, il * S, SB_NONE, 0, OUT_ADD, last, 1));
    const int io = nd - 2 - q;  // the other strips' line
    if (io >= 0) ts.push_back(task({term(iH + io, SB_V, (io + 1) * S, 1)}, SB_V, io * S, SB_NONE, 0, OUT_ADD, 0, nl));
    prog.push_back(group(ts));
  }
  for (int l = d; l >= 1; --l) {
    const int h = 1 << (l - 1), src = l == 1 ? SB_RIN : SB_W;
    const int lev = bd.iLev + 5 * (l - 1), Dinv = lev, P = lev + 3, Q = lev + 4;
    std::vector<GTask> ts;
    for (int p = h; p < R - h; p += 2 * h)
      ts.push_back(task({term(Dinv, src, p, 0), term(P, SB_V, p - h, 1), term(Q, SB_V, p + h, 1)}, SB_V, p,
                        SB_NONE, 0, OUT_SET, 0, N));
    ts.push_back(task({term(Dinv, src, R - h, 0), term(P, SB_V, R - 2 * h, 1)}, SB_V, R - h, SB_NONE, 0, OUT_SET, 0,
                      nl));
    ts.push_back(task({term(Dinv, src, R - h, 0), term(P, SB_V, R - 2 * h, 1), term(Q, SB_V, R, 1)}, SB_V, R - h,
                      SB_NONE, 0, OUT_SET, last, 1));
    prog.push_back(group(ts));
  }
}

// The double sweep with the interface data passed by scans and the interior corrections as
// single grouped steps (form 1):
//   F1  w_s = D^{-1} r_s, every strip at once (block Thomas steps, as in build_steps);
//   F2  t_s = w_s[R-1] - G t_{s-1} (s = 0..N-2, t_{-1} = 0) as a prefix-doubling scan:
//       a^0_s = w_s[R-1], a^{l+1}_s = a^l_s + (-G)^(2^l) a^l_{s-2^l} (ceil(log2(N-1)) steps,
//       every strip in each step, ping-pong between T0 and T1);
//   F3  v_s[j] = w_s[j] - Y_j t_{s-1}, every line j of strips 1..N-1 in one step, with the block
//       columns Y_j = D^{-1}[j, 0] L of the strip inverse (D of the strips before the last,
//       or of the last one); v_s[R-1] = t_s follows for the strips before the last;
//   B1  u_s[0] = v_s[0] - K u_{s+1}[0] (s = N-2..0, u_{N-1}[0] = v_{N-1}[0]) as a scan with
//       (-K)^(2^l) and strip offsets +2^l (ceil(log2 N) steps), then copied into V's line 0;
//   B2  u_s[j] = v_s[j] - Z_j u_{s+1}[0], lines j = 1..R-1 of strips 0..N-2 in one step,
//       Z_j = D^{-1}[j, R-1] U.
// Every step is exact algebra on the block-Thomas form; only the order of the sums differs.
// F1 by the twisted block factorisation of the strip matrix D of lines 0..R-1 (the same in
// every strip; the last strip's extra line R follows after F3, see build_program): with the
// block-Thomas factors F_j from the top, G_j from the bottom and M at line q (BlockDir),
//   forward, step i = 0, 1, ..: the top line j = i < q,       y_j = F_j (r_j - L y_{j-1}),
//                               the bottom line j = R-1-i > q, z_j = G_j (r_j - U z_{j+1});
//   middle:                     x_q = M (r_q - L y_{q-1} - U z_{q+1});
//   back, step i = 0, 1, ..:    x_j = y_j - F_j U x_{j+1} (j = q-1-i),
//                               x_j = z_j - G_j L x_{j-1} (j = q+1+i).
// Both ends advance in one grouped step (two tasks over all strips), so the dependent chain
// is 2 max(q, R-1-q) + 1 steps instead of block Thomas's 2R - 1, with the same factor bytes.
// Every line j of V holds y_j (j < q) or z_j (j > q) until the back substitution overwrites it.
static void append_twisted_f1(std::vector<SweepPhase>& prog, int R, int N, const BlockDir& bd) {
  const int q = bd.twq;
  auto coupled = [](int f, int line, int cpl, int bline) {
    // x = Rin[bline] - C(V[line]) (bline < 0: no base)
    GTerm g{f, SB_V, line, 0, 1, cpl, bline >= 0 ? SB_RIN : 0, bline >= 0 ? bline : 0};
    return g;
  };
  auto task = [&](std::initializer_list<GTerm> terms, int out_line, int mode) {
    GTask t{};
    t.nterm = 0;
    for (const GTerm& g : terms) t.term[t.nterm++] = g;
    t.out_arr = SB_V; t.out_line = out_line;
    t.base_arr = SB_NONE; t.base_line = 0;
    t.mode = mode; t.s0 = 0; t.ns = N;
    return t;
  };
  const int half = std::max(q, R - 1 - q);
  for (int i = 0; i < half; ++i) {
    SweepPhase p;
    p.kind = PH_GROUP;
    if (i < q) {
      const int j = i;
      p.tasks.push_back(j == 0 ? task({GTerm{0, SB_RIN, 0, 0, 0, 0, 0, 0}}, 0, OUT_SET)
                               : task({coupled(j, j - 1, XC_LOWER, j)}, j, OUT_SET));
    }
    if (R - 1 - i > q) {
      const int j = R - 1 - i, f = bd.iTw + j - q - 1;
      p.tasks.push_back(j == R - 1 ? task({GTerm{f, SB_RIN, j, 0, 0, 0, 0, 0}}, j, OUT_SET)
                                   : task({coupled(f, j + 1, XC_UPPER, j)}, j, OUT_SET));
    }
    prog.push_back(p);
  }
  {
    SweepPhase p;
    p.kind = PH_GROUP;
    p.tasks.push_back(task({coupled(bd.iTwM, q - 1, XC_LOWER, q), coupled(bd.iTwM, q + 1, XC_UPPER, -1)}, q, OUT_SET));
    prog.push_back(p);
  }
  for (int i = 0; i < half; ++i) {
    SweepPhase p;
    p.kind = PH_GROUP;
    if (q - 1 - i >= 0) {
      const int j = q - 1 - i;
      p.tasks.push_back(task({coupled(j, j + 1, XC_UPPER, -1)}, j, OUT_ADD));
    }
    if (q + 1 + i <= R - 1) {
      const int j = q + 1 + i;
      p.tasks.push_back(task({coupled(bd.iTw + j - q - 1, j - 1, XC_LOWER, -1)}, j, OUT_ADD));
    }
    prog.push_back(p);
  }
}

std::vector<SweepPhase> build_program(int n, int N, bool double_sweep, int form, const BlockDir& bd, int depth) {
  std::vector<SweepPhase> prog;
  const int R = n / N;
  auto as_step = [](const SweepStep& x) {
    SweepPhase p;
    p.kind = PH_STEP;
    p.step = x;
    return p;
  };
  const std::vector<SweepStep> legacy = build_steps(n, N, double_sweep);
  const bool twisted = depth == PROG_TWISTED;
  if (twisted) append_twisted_f1(prog, R, N, bd);
  else if (depth > 0) append_bcr_f1(prog, R, N, depth, bd);
  else
    for (int q = 0; q < 2 * R + 1; ++q) prog.push_back(as_step(legacy[q]));  // F1
  if (form == 0 || N < 2) {
    for (size_t q = 2 * R + 1; q < legacy.size(); ++q) prog.push_back(as_step(legacy[q]));
    return prog;
  }
  auto task1 = [](int f, int arr, int line, int ds, int neg, int out_arr, int out_line, int base_arr, int base_line,
                  int mode, int s0, int ns) {
    GTask t{};
    t.nterm = 1;
    t.term[0] = GTerm{f, arr, line, ds, neg, 0, 0, 0};
    t.out_arr = out_arr; t.out_line = out_line;
    t.base_arr = base_arr; t.base_line = base_line;
    t.mode = mode; t.s0 = s0; t.ns = ns;
    return t;
  };
  const int FG = R + 1, FK = R + 2;
  // F2.  With the twisted strip solves and R even, the top chain is one step longer than the
  // bottom one: line R-1, all the scan reads, is final a step before line 0, so the first scan
  // step joins that last step of F1 (two tasks on disjoint lines) instead of following it.
  const bool join_first = twisted && bd.LF > 0 && !prog.empty() && prog.back().kind == PH_GROUP &&
                          prog.back().tasks.size() == 1 && prog.back().tasks[0].out_line == 0 && R - 1 > 1;
  int src_arr = SB_V, src_line = R - 1;
  for (int l = 0; l < bd.LF; ++l) {
    SweepPhase p;
    p.kind = PH_GROUP;
    const int dst = (l & 1) ? SB_T1 : SB_T0;
    p.tasks.push_back(task1(l == 0 ? FG : bd.iGp + l - 1, src_arr, src_line, -(1 << l), l == 0 ? 1 : 0, dst, 0,
                            src_arr, src_line, OUT_SET, 0, N - 1));
    if (l == 0 && join_first) prog.back().tasks.push_back(p.tasks[0]);
    else prog.push_back(p);
    src_arr = dst;
    src_line = 0;
  }
  // F3
  if (twisted) {
    // F1 solved the first R lines of the last strip like every other strip, so its first-line
    // correction uses the same Y_j; then its extra line R by the Schur complement of lines
    // 0..R-1, whose inverse is F_R: x_R = F_R (r_R - L v[R-1]), and x_j = v[j] - Z_j x_R with
    // Z_j = D_int^{-1}[j, R-1] U (the coupling of line R-1 to line R)
    SweepPhase p;
    p.kind = PH_GROUP;
    for (int j = 0; j < R; ++j)
      p.tasks.push_back(task1(bd.iY + j, src_arr, src_line, -1, 1, SB_V, j, SB_NONE, 0, OUT_ADD, 1, N - 1));
    prog.push_back(p);
    prog.push_back(as_step(legacy[R]));
    SweepPhase c;
    c.kind = PH_GROUP;
    for (int j = 0; j < R; ++j)
      c.tasks.push_back(task1(j == 0 ? bd.iZ0 : bd.iZ + j - 1, SB_V, R, 0, 1, SB_V, j, SB_NONE, 0, OUT_ADD, N - 1, 1));
    prog.push_back(c);
  } else {
    SweepPhase p;
    p.kind = PH_GROUP;
    if (N >= 3)
      for (int j = 0; j < R; ++j)
        p.tasks.push_back(task1(bd.iY + j, src_arr, src_line, -1, 1, SB_V, j, SB_NONE, 0, OUT_ADD, 1, N - 2));
    for (int j = 0; j <= R; ++j)
      p.tasks.push_back(task1(bd.iYL + j, src_arr, src_line, -1, 1, SB_V, j, SB_NONE, 0, OUT_ADD, N - 1, 1));
    prog.push_back(p);
  }
  if (!double_sweep) return prog;
  // B1
  src_arr = SB_V;
  src_line = 0;
  for (int l = 0; l < bd.LB; ++l) {
    SweepPhase p;
    p.kind = PH_GROUP;
    const int dst = (l & 1) ? SB_T1 : SB_T0;
    p.tasks.push_back(task1(l == 0 ? FK : bd.iKp + l - 1, src_arr, src_line, 1 << l, l == 0 ? 1 : 0, dst, 0, src_arr,
                            src_line, OUT_SET, 0, N));
    prog.push_back(p);
    src_arr = dst;
    src_line = 0;
  }
  // B2, then u_s[0] into V's line 0
  {
    SweepPhase p;
    p.kind = PH_GROUP;
    for (int j = 1; j < R; ++j)
      p.tasks.push_back(task1(bd.iZ + j - 1, src_arr, 0, 1, 1, SB_V, j, SB_NONE, 0, OUT_ADD, 0, N - 1));
    if (!p.tasks.empty()) prog.push_back(p);
    SweepPhase c;
    c.kind = PH_COPY;
    c.tasks.push_back(task1(0, src_arr, 0, 0, 0, SB_V, 0, SB_NONE, 0, OUT_SET, 0, N - 1));
    prog.push_back(c);
  }
  return prog;
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

// X[j][i][s][c] <- scale * src (frame-mapped); entries (j = R, s < N-1) are padding (zero).
template <typename R>
__global__ void pack_kernel(const double2* const* __restrict__ srcptr, const double* __restrict__ scale, int C,
                            int t, int4 codes, int n, int N, int Rl, typename Cx<R>::T* __restrict__ X) {
  using T = typename Cx<R>::T;
  const int m = n + 1;
  const size_t total = (size_t)(Rl + 1) * m * N * C;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % C);
    size_t q = idx / C;
    const int s = (int)(q % N);
    q /= N;
    const int i = (int)(q % m);
    const int j = (int)(q / m);
    T v = mk<T>(0, 0);
    if (j < Rl || s == N - 1) {
      int io, jo;
      frame_map(code_of(codes, c % t), i, s * Rl + j, n, io, jo);
      const double2 a = srcptr[c][(size_t)jo * m + io];
      const double sc = scale[c];
      v = mk<T>(a.x * sc, a.y * sc);
    }
    X[idx] = v;
  }
}

template <typename R>
__global__ void unpack_kernel(const typename Cx<R>::T* __restrict__ X, int C, int t, int4 codes, int n, int N, int Rl,
                              double2* __restrict__ dst, size_t stride) {
  const int m = n + 1;
  const size_t total = (size_t)(Rl + 1) * m * N * C;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % C);
    size_t q = idx / C;
    const int s = (int)(q % N);
    q /= N;
    const int i = (int)(q % m);
    const int j = (int)(q / m);
    if (j == Rl && s != N - 1) continue;
    int io, jo;
    frame_map(code_of(codes, c % t), i, s * Rl + j, n, io, jo);
    dst[(size_t)c * stride + (size_t)jo * m + io] = to_d(X[idx]);
  }
}

// Same as unpack_kernel with one destination pointer per column.
template <typename R>
__global__ void unpack_tab_kernel(const typename Cx<R>::T* __restrict__ X, int C, int t, int4 codes, int n, int N,
                                  int Rl, double2* const* __restrict__ dstcol) {
  const int m = n + 1;
  const size_t total = (size_t)(Rl + 1) * m * N * C;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % C);
    size_t q = idx / C;
    const int s = (int)(q % N);
    q /= N;
    const int i = (int)(q % m);
    const int j = (int)(q / m);
    if (j == Rl && s != N - 1) continue;
    int io, jo;
    frame_map(code_of(codes, c % t), i, s * Rl + j, n, io, jo);
    dstcol[c][(size_t)jo * m + io] = to_d(X[idx]);
  }
}

// Narrow step (at most 8 columns: the interface chains and the last strip's extra line
// of a single right-hand side).  The CTA forms x (m x ncols) in shared memory, column-major
// so that the 32 lanes of a warp read 32 consecutive node indices of one column without bank
// conflicts; then one warp per output row walks the row of A (consecutive entries per lane,
// eight loads in flight) and sums across the warp with shuffles.
template <typename R>
__global__ void __launch_bounds__(256) line_gemv_kernel(const typename Cx<R>::T* __restrict__ A, int lda, int m,
                                                        LineOperand<typename Cx<R>::T> op, Coef cf) {
  using T = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);
  const int ncols = op.ns * op.C;
  const int N = op.N, C = op.C;
  const double2 ve = cf.vert(0), vi = cf.vert(1);
  const T vert_edge = mk<T>(ve.x, ve.y), vert_int = mk<T>(vi.x, vi.y);
  const R dg = (R)cf.diag();
  const int total = m * ncols;
  // x: every thread first loads all its inputs, then forms its entries
  constexpr int PT = 8;  // entries per thread per pass
  for (int base_idx = threadIdx.x * PT; base_idx < total; base_idx += blockDim.x * PT) {
    T b[PT], s0[PT], s1[PT];
#pragma unroll
    for (int u = 0; u < PT; ++u) {
      const int idx = base_idx + u;
      b[u] = s0[u] = s1[u] = mk<T>(0, 0);
      if (idx >= total) continue;
      const int i = idx / ncols, col = idx % ncols;
      const int s = op.s0 + col / C, c = col % C;
      if (op.base) b[u] = op.base[((size_t)(op.base_j * m + i) * N + s) * C + c];
      if (op.cpl != XC_NONE) {
        const T* sp = op.src + ((size_t)op.src_j * m * N + (s + op.src_ds)) * C + c;
        const size_t istride = (size_t)N * C;
        s0[u] = __ldcg(sp + (size_t)i * istride);
        const int nb = (op.cpl == XC_LOWER) ? i - 1 : i + 1;
        if (op.cpl != XC_IDENT && nb >= 0 && nb < m) s1[u] = __ldcg(sp + (size_t)nb * istride);
      }
    }
#pragma unroll
    for (int u = 0; u < PT; ++u) {
      const int idx = base_idx + u;
      if (idx >= total) continue;
      T v = b[u];
      if (op.cpl != XC_NONE) {
        T cp = s0[u];
        if (op.cpl != XC_IDENT) {
          const int i = idx / ncols;
          cp = cmul((i == 0 || i == m - 1) ? vert_edge : vert_int, cp);
          cp.x += dg * s1[u].x;
          cp.y += dg * s1[u].y;
        }
        v = op.neg ? csub(v, cp) : cadd(v, cp);
      }
      xs[(idx % ncols) * m + idx / ncols] = v;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int row = blockIdx.x * 8 + wid;
  if (row >= m) return;
  T acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = mk<T>(0, 0);
  const T* Ar = A + (size_t)row * lda;
  constexpr int U = 8;  // loads in flight per lane
  for (int k0 = lane; k0 < m; k0 += 32 * U) {
    T a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + 32 * u;
      a[u] = k < m ? __ldg(Ar + k) : mk<T>(0, 0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + 32 * u;
      if (k < m) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (c < ncols) cfma(acc[c], a[u], xs[c * m + k]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 8; ++c)
#pragma unroll
    for (int o = 16; o; o >>= 1) acc[c] = cadd(acc[c], shfl_xor(acc[c], o));
  if (lane < ncols) {
    T z = acc[0];
#pragma unroll
    for (int c = 1; c < 8; ++c)
      if (lane == c) z = acc[c];
    const int s = op.s0 + lane / C, c = lane % C;
    T* o = op.out + ((size_t)(op.out_j * m + row) * N + s) * C + c;
    apply_out(o, z, op.out_mode);
    if (op.acc) {
      T* a2 = op.acc + ((size_t)(op.acc_j * m + row) * N + s) * C + c;
      apply_out(a2, op.out_mode == OUT_SET ? z : *o, op.acc_mode);
    }
  }
}

// Narrow steps, second form: x (m x ncols, ncols <= 8) is formed once into a column-major
// scratch array xout[c * m + k] by line_xbuild_kernel; line_gemv_split_kernel then gives
// each CTA RPC rows of the factor block and splits the node index across its 8 warps, so that
// every lane issues its loads of A and x together; the warps' partial sums meet in shared
// memory before the step's output modes.
template <typename R>
__global__ void line_xbuild_kernel(int m, LineOperand<typename Cx<R>::T> op, Coef cf, typename Cx<R>::T* __restrict__ xout) {
  using T = typename Cx<R>::T;
  const int ncols = op.ns * op.C, N = op.N, C = op.C;
  const size_t istride = (size_t)N * C;
  const double2 ve = cf.vert(0), vi = cf.vert(1);
  const T vert_edge = mk<T>(ve.x, ve.y), vert_int = mk<T>(vi.x, vi.y);
  const R dg = (R)cf.diag();
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * ncols; idx += gridDim.x * blockDim.x) {
    const int k = idx / ncols, col = idx % ncols;
    const int s = op.s0 + col / C, c = col % C;
    T v = op.base ? __ldcg(op.base + ((size_t)(op.base_j * m + k) * N + s) * C + c) : mk<T>(0, 0);
    if (op.cpl != XC_NONE) {
      const T* sp = op.src + ((size_t)op.src_j * m * N + (s + op.src_ds)) * C + c;
      T cp = __ldcg(sp + (size_t)k * istride);
      if (op.cpl != XC_IDENT) {
        const int nb = op.cpl == XC_LOWER ? k - 1 : k + 1;
        const T y = (nb >= 0 && nb < m) ? __ldcg(sp + (size_t)nb * istride) : mk<T>(0, 0);
        cp = cmul((k == 0 || k == m - 1) ? vert_edge : vert_int, cp);
        cp.x += dg * y.x;
        cp.y += dg * y.y;
      }
      v = op.neg ? csub(v, cp) : cadd(v, cp);
    }
    xout[(size_t)col * m + k] = v;
  }
}

template <typename R, int RPC>
__global__ void __launch_bounds__(256) line_gemv_split_kernel(const typename Cx<R>::T* __restrict__ A, int lda, int m,
                                                              LineOperand<typename Cx<R>::T> op,
                                                              const typename Cx<R>::T* __restrict__ x) {
  using T = typename Cx<R>::T;
  __shared__ T red[8][RPC][8];
  const int ncols = op.ns * op.C;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * RPC;
  const int kw = ((m + 7) / 8 + 31) / 32 * 32;  // node indices per warp, a multiple of 32
  const int kb = warp * kw, ke = min(m, kb + kw);
  T acc[RPC][8];
#pragma unroll
  for (int r = 0; r < RPC; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = mk<T>(0, 0);
#pragma unroll 2
  for (int k = kb + lane; k < ke; k += 32) {
    T a[RPC];
#pragma unroll
    for (int r = 0; r < RPC; ++r) a[r] = row0 + r < m ? __ldg(A + (size_t)(row0 + r) * lda + k) : mk<T>(0, 0);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c < ncols) {
        const T xv = __ldcg(x + (size_t)c * m + k);
#pragma unroll
        for (int r = 0; r < RPC; ++r) cfma(acc[r][c], a[r], xv);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RPC; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c < ncols) {
        T v = acc[r][c];
#pragma unroll
        for (int o = 16; o; o >>= 1) v = cadd(v, shfl_xor(v, o));
        if (lane == 0) red[warp][r][c] = v;
      }
    }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < RPC * ncols) {
    const int r = t / ncols, col = t % ncols;
    const int gr = row0 + r;
    if (gr < m) {
      T z = red[0][r][col];
#pragma unroll
      for (int w = 1; w < 8; ++w) z = cadd(z, red[w][r][col]);
      const int N = op.N, C = op.C;
      const int s = op.s0 + col / C, c = col % C;
      T* o = op.out + ((size_t)(op.out_j * m + gr) * N + s) * C + c;
      apply_out(o, z, op.out_mode);
      if (op.acc) {
        T* a2 = op.acc + ((size_t)(op.acc_j * m + gr) * N + s) * C + c;
        apply_out(a2, op.out_mode == OUT_SET ? z : *o, op.acc_mode);
      }
    }
  }
}

// Interface chains (F2 and B1 above): L narrow steps y_{s_q} (op) M x, x = line src_j of strip
// s_q + src_ds, where strip s_q + src_ds is the one step q-1 wrote (s_q = s_0 + q dir,
// dir = -src_ds).  One cooperative launch runs the whole chain: every CTA copies its rows of M
// into shared memory once and keeps them for all L steps, and a grid barrier separates the
// steps, in place of two launches (x build, GEMV) per step that each re-read M.
template <typename T>
struct ChainOp {
  const T* src;
  T* out;
  int src_j, out_j, s0, dir, src_ds, L, out_mode, N, C;
};

template <typename R, int CMAX>
__global__ void __launch_bounds__(1024) chain_kernel(const typename Cx<R>::T* __restrict__ A, int lda, int m,
                                                     ChainOp<typename Cx<R>::T> op, unsigned* bar, int* err,
                                                     long long budget) {
  using T = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rows = (m + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * rows, nr = max(0, min(m, r0 + rows) - r0);
  const int C = op.C, N = op.N;
  const int nwarp = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // warps per row: each takes a contiguous slice of the nodes, a multiple of 32 long
  const int ks = max(1, nwarp / rows);
  const int kspan = ((m + ks - 1) / ks + 31) / 32 * 32;
  const int lr = warp / ks, kq = warp % ks;
  T* Ms = reinterpret_cast<T*>(smem_raw);  // rows x m: this CTA's rows of M
  T* xs = Ms + (size_t)rows * m;           // C x m, column-major (lanes read consecutive nodes)
  T* part = xs + (size_t)m * C;            // rows x ks x C partial sums of the warps
  T* cur0 = part + (size_t)rows * ks * CMAX;  // 2 x (rows x C): the step's output lines, by step parity
  for (int r = 0; r < nr; ++r)
#pragma unroll 2
    for (int k = threadIdx.x; k < m; k += blockDim.x) Ms[(size_t)r * m + k] = __ldg(A + (size_t)(r0 + r) * lda + k);
  unsigned target = 0;
  for (int q = 0; q < op.L; ++q) {
    const int s = op.s0 + q * op.dir, sx = s + op.src_ds;
    // the output lines of this step are not written by the chain's earlier steps: fetch them
    // before the barrier (the buffer of this parity was last read two steps ago, before the
    // barrier that ended step q - 1 began)
    T* cur = cur0 + (q & 1) * rows * C;
    if (threadIdx.x < nr * C) {
      const int r = threadIdx.x / C, c = threadIdx.x - r * C;
      cur[threadIdx.x] = __ldcg(op.out + ((size_t)(op.out_j * m + r0 + r) * N + s) * C + c);
    }
    // step q - 1 wrote the line read now: every CTA's rows of it must be in place
    if (q > 0 && !grid_sync(bar, target, err, budget)) return;
    const T* xsrc = op.src + ((size_t)op.src_j * m * N + sx) * C;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
      T v[CMAX];
#pragma unroll
      for (int c = 0; c < CMAX; ++c)
        if (c < C) v[c] = __ldcg(xsrc + (size_t)k * N * C + c);
#pragma unroll
      for (int c = 0; c < CMAX; ++c)
        if (c < C) xs[(size_t)c * m + k] = v[c];
    }
    __syncthreads();
    if (lr < nr) {
      T acc[CMAX];
#pragma unroll
      for (int c = 0; c < CMAX; ++c) acc[c] = mk<T>(0, 0);
      const T* mrow = Ms + (size_t)lr * m;
      const int kb = kq * kspan, ke = min(m, kb + kspan);
#pragma unroll 2
      for (int k = kb + lane; k < ke; k += 32) {
        const T a = mrow[k];
#pragma unroll
        for (int c = 0; c < CMAX; ++c)
          if (c < C) cfma(acc[c], a, xs[(size_t)c * m + k]);
      }
#pragma unroll
      for (int c = 0; c < CMAX; ++c) {
        if (c < C) {
          T v = acc[c];
#pragma unroll
          for (int o = 16; o; o >>= 1) v = cadd(v, shfl_xor(v, o));
          if (lane == 0) part[((size_t)lr * ks + kq) * CMAX + c] = v;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < nr * C) {
      const int r = threadIdx.x / C, c = threadIdx.x - r * C;
      T z = part[(size_t)r * ks * CMAX + c];
      for (int j = 1; j < ks; ++j) z = cadd(z, part[((size_t)r * ks + j) * CMAX + c]);
      T* o = op.out + ((size_t)(op.out_j * m + r0 + r) * N + s) * C + c;
      const T c0 = cur[threadIdx.x];
      *o = op.out_mode == OUT_SET ? z : (op.out_mode == OUT_SUB ? csub(c0, z) : cadd(c0, z));
    }
  }
}

// bf16 factor products keep block Thomas: the bottom-up factors G_j belong to sub-strips whose
// ends are both cut (no absorbing line), their norms are larger, and with 8-bit factor entries
// the twisted sweep erred 8 times as much as block Thomas on 45-line strips (6.3 against
// 0.76 per cent); in complex64 both stay within the same bar.
bool Engine::twisted_ok(int C) const {
  return bdir.iTw >= 0 && precision == HH_PREC_FP32 && !lowp && tc_ready && C % 2 == 0 &&
         !prog_double_d[PROG_TWISTED].empty();
}

int Engine::depth_for(int C) const {
  const auto it = bcr_tuned.find(C);
  if (it != bcr_tuned.end()) return it->second;
  if (opts.bcr_depth > 0) return opts.bcr_depth;  // an explicit depth before the default
  if (opts.twisted == 1 && twisted_ok(C)) return PROG_TWISTED;
  return 0;
}

const std::vector<SweepPhase>& Engine::program(int C, bool single) const {
  const int d = depth_for(C);
  return single ? prog_single_d[d] : prog_double_d[d];
}

int Engine::upload_programs() {
  std::vector<GTask> all;
  for (int d = 0; d < NPROG; ++d)
    for (std::vector<SweepPhase>* prog : {&prog_double_d[d], &prog_single_d[d]})
      for (SweepPhase& ph : *prog) {
        ph.dev_off = all.size();
        for (const GTask& t : ph.tasks) all.push_back(t);
      }
  dfree(prog_tasks);
  prog_tasks = nullptr;
  if (all.empty()) return HH_OK;
  if (dmalloc((void**)&prog_tasks, all.size() * sizeof(GTask))) return HH_ENOMEM;
  cudaMemcpy(prog_tasks, all.data(), all.size() * sizeof(GTask), cudaMemcpyHostToDevice);
  return HH_OK;
}

size_t Engine::sweep_ws_bytes(int C) const { return (size_t)(R + 1) * m * N * C * sweep_elem(); }

size_t Engine::sweep_partial_bytes(int C) const { return (size_t)8 * m * N * C * sweep_elem(); }

int Engine::ensure_sweep_ws(int C) {
  if ((size_t)C <= w_cap_cols) return HH_OK;
  dfree(w_rin); dfree(w_v); dfree(w_w); dfree(w_partial); dfree(w_t0); dfree(w_t1);
  w_rin = w_v = w_w = w_partial = w_t0 = w_t1 = nullptr;
  w_cap_cols = 0;
  w_partial_bytes = 0;
  const size_t b = sweep_ws_bytes(C), bt = (size_t)m * N * C * sweep_elem();
  if (dmalloc(&w_rin, b) || dmalloc(&w_v, b) || dmalloc(&w_w, b) || dmalloc(&w_partial, sweep_partial_bytes(C)) ||
      dmalloc(&w_t0, bt) || dmalloc(&w_t1, bt))
    return HH_ENOMEM;
  w_partial_bytes = sweep_partial_bytes(C);
  w_cap_cols = C;
  return HH_OK;
}

// Algorithmic bytes of one step: it reads its m x m block and its input lines once and
// writes its output (and accumulated) lines once.
static double step_bytes(const Engine& E, const SweepStep& s, int C) {
  const double e = (double)E.sweep_elem();
  const double line = (double)E.m * s.ns * C * e;
  return (double)E.m * E.m * e + line * ((s.base != SB_NONE) + (s.src != SB_NONE) + 1 + 2 * (s.acc != SB_NONE) +
                                         (s.out_mode != OUT_SET));
}

// One wide step on the tensor cores with tile shape CF and K split nsplit_req (0: split until
// the SMs are filled); the K slices meet in split_reduce_kernel.
template <class CF>
static cudaError_t launch_tc_step(Engine& E, const LineOperand<float2>& op, int fblock, int C, int nsplit_req,
                                  const void* Rin, void* partial_buf, size_t partial_bytes, bool cluster = false) {
  const int ncols = op.ns * C;
  const int gx = (E.m + tc::BM - 1) / tc::BM, gy = (ncols + CF::BNC - 1) / CF::BNC;
  int nsplit = nsplit_req > 0 ? nsplit_req : std::max(1, std::min(8, (E.num_sms - 4) / (gx * gy)));
  if (!cluster)
    while (nsplit > 1 && (size_t)nsplit * E.m * ncols * sizeof(float2) > partial_bytes) --nsplit;
  const int kchunk = ((E.m + nsplit - 1) / nsplit + tc::BKC - 1) / tc::BKC * tc::BKC;
  nsplit = (E.m + kchunk - 1) / kchunk;  // no empty split
  // the maps are copied out at once: the second lookup may evict the first one's ring slot
  CUtensorMap map_base, map_src;
  {
    const Engine::LineMaps* mb = E.line_maps_for(op.base ? op.base : Rin, C, CF::BNC);
    if (!mb) return cudaErrorInvalidValue;
    map_base = mb->base;
    const Engine::LineMaps* ms = E.line_maps_for(op.src ? op.src : Rin, C, CF::BNC);
    if (!ms) return cudaErrorInvalidValue;
    map_src = ms->src;
  }
  // launch attributes: the K slices of a tile as one cluster (they meet in distributed shared
  // memory), and programmatic dependent launch (the step's prologue and first factor tiles
  // overlap the end of the preceding kernel; the kernel waits for it before touching the
  // line data)
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(gx, gy, nsplit);
  cfg.blockDim = dim3(tc::THREADS);
  cfg.dynamicSmemBytes = CF::SMEM;
  cfg.stream = E.stream;
  cudaLaunchAttribute attr[2];
  unsigned na = 0;
  const bool in_cluster = cluster && nsplit > 1;
  if (in_cluster && nsplit > 8) return cudaErrorInvalidValue;  // the kernel sums at most 8 slices
  if (in_cluster) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = 1;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = nsplit;
    ++na;
  }
  if (E.opts.overlap_steps) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  if (in_cluster) {
    float2* nopartial = nullptr;
    const cudaError_t ce =
        cudaLaunchKernelEx(&cfg, tc_line_gemm_kernel<CF, true>, E.tmap_hi, E.tmap_lo, map_base, map_src, fblock, E.m,
                           op, E.coef, kchunk, nopartial, E.err, E.opts.timeout_cycles);
    E.count_launch();
    return ce;
  }
  float2* partial = nsplit > 1 ? reinterpret_cast<float2*>(partial_buf) : nullptr;
  const cudaError_t ce =
      cudaLaunchKernelEx(&cfg, tc_line_gemm_kernel<CF, false>, E.tmap_hi, E.tmap_lo, map_base, map_src, fblock, E.m,
                         op, E.coef, kchunk, partial, E.err, E.opts.timeout_cycles);
  E.count_launch();
  if (ce != cudaSuccess) return ce;
  if (nsplit > 1) {
    // also with programmatic dependent launch: its CTAs wait, resident, for the step to
    // complete, and the next step's CTAs start their prologue while it runs
    cudaLaunchConfig_t rc{};
    rc.gridDim = dim3(E.grid_for((size_t)E.m * ncols));
    rc.blockDim = dim3(256);
    rc.stream = E.stream;
    cudaLaunchAttribute ra[1];
    ra[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    ra[0].val.programmaticStreamSerializationAllowed = 1;
    rc.attrs = ra;
    rc.numAttrs = E.opts.overlap_steps ? 1 : 0;
    const cudaError_t re = cudaLaunchKernelEx(&rc, split_reduce_kernel<float>, (const float2*)partial, nsplit, E.m, op);
    E.count_launch();
    if (re != cudaSuccess) return re;
  }
  return cudaSuccess;
}

// tile shapes of the autotuner: 0 = 64, 1 = 32, 2 = 128 complex columns per CTA
static constexpr int kTcShapes = 3;
static cudaError_t launch_tc_shape(Engine& E, int shape, const LineOperand<float2>& op, int fblock, int C,
                                   int nsplit_req, const void* Rin, void* partial_buf, size_t partial_bytes,
                                   bool cluster) {
  if (shape == 1) return launch_tc_step<tc::Narrow>(E, op, fblock, C, nsplit_req, Rin, partial_buf, partial_bytes, cluster);
  if (shape == 2) return launch_tc_step<tc::Huge>(E, op, fblock, C, nsplit_req, Rin, partial_buf, partial_bytes, cluster);
  return launch_tc_step<tc::Wide>(E, op, fblock, C, nsplit_req, Rin, partial_buf, partial_bytes, cluster);
}

template <typename R>
static cudaError_t run_steps_t(Engine& E, const std::vector<SweepStep>& steps, const GArrays& arrs, int C,
                               void* partial_buf, size_t partial_bytes, bool allow_tick) {
  using T = typename Cx<R>::T;
  const void* Rin = arrs.p[SB_RIN];
  const T* Fb = reinterpret_cast<const T*>(E.factors);
  const size_t blk = (size_t)E.m * E.ldf;
  auto buf = [&](int b) -> T* { return b == SB_NONE ? nullptr : reinterpret_cast<T*>(arrs.p[b]); };
  const size_t gemv_cap = 200 * 1024;  // the narrow kernel keeps x (m x ncols) in shared memory
  constexpr int BM = 64, BN = 64, BK = 16, STG = 3;
  constexpr size_t gemm_smem = line_gemm_smem<R, BM, BN, BK, STG>();
  auto gemm_fn = line_gemm_kernel<R, BM, BN, BK, 4, 4, STG>;
  cudaFuncSetAttribute((const void*)gemm_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem);
  cudaFuncSetAttribute((const void*)line_gemv_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)std::min<size_t>((size_t)E.m * 8 * sizeof(T), gemv_cap));
  // allow_tick: time the wide GEMM steps one by one (a sampled, eager sweep)
  const bool tick_gemm = allow_tick && E.opts.profile;
  // interface chains: one cooperative launch per run of chained narrow steps
  constexpr int chain_threads = 1024;
  const int chain_grid = E.num_sms;
  const int chain_rows = (E.m + chain_grid - 1) / chain_grid;
  const int chain_ks = std::max(1, (chain_threads / 32) / chain_rows);
  const size_t chain_smem = ((size_t)chain_rows * E.m + (size_t)E.m * C + (size_t)chain_rows * chain_ks * 8 +
                             2 * (size_t)chain_rows * C) * sizeof(T);
  int chain_fit = 0;
  const void* chain_fn = C <= 4 ? (const void*)chain_kernel<R, 4> : (const void*)chain_kernel<R, 8>;
  if (E.opts.fuse_chains && C <= 8 && chain_rows <= chain_threads / 32 && chain_rows * C <= chain_threads &&
      chain_smem <= 220 * 1024) {
    cudaFuncSetAttribute(chain_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chain_smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&chain_fit, chain_fn, chain_threads, chain_smem);
  }
  auto chainable = [](const SweepStep& x) {
    return x.ns == 1 && x.cpl == XC_IDENT && !x.neg && x.base == SB_NONE && x.acc == SB_NONE && x.src_ds != 0 &&
           x.src == x.out && x.src_j == x.out_j;
  };
  for (size_t si = 0; si < steps.size(); ++si) {
    const SweepStep& s = steps[si];
    if (chain_fit >= 1 && chainable(s)) {
      const int dir = -s.src_ds;
      size_t L = 1;
      while (si + L < steps.size()) {
        const SweepStep& u = steps[si + L];
        if (!chainable(u) || u.f != s.f || u.src != s.src || u.src_j != s.src_j || u.src_ds != s.src_ds ||
            u.out_mode != s.out_mode || u.s0 != s.s0 + (int)L * dir)
          break;
        ++L;
      }
      if (L >= 2) {
        ChainOp<T> cop{};
        cop.src = buf(s.src); cop.out = buf(s.out);
        cop.src_j = s.src_j; cop.out_j = s.out_j; cop.s0 = s.s0; cop.dir = dir; cop.src_ds = s.src_ds;
        cop.L = (int)L; cop.out_mode = s.out_mode; cop.N = E.N; cop.C = C;
        const T* A = Fb + (size_t)s.f * blk;
        unsigned* cbar = E.bar + Engine::BAR_CHAIN * GRID_BAR_WORDS;
        cudaMemsetAsync(cbar, 0, GRID_BAR_WORDS * sizeof(unsigned), E.stream);
        int lda = E.ldf, mm = E.m;
        void* args[] = {(void*)&A, (void*)&lda, (void*)&mm, (void*)&cop, (void*)&cbar, (void*)&E.err,
                        (void*)&E.opts.timeout_cycles};
        const cudaError_t ce = E.launch_coop(chain_fn, chain_grid, chain_threads, chain_smem, args);
        if (ce != cudaSuccess) return ce;
        si += L - 1;
        continue;
      }
    }
    LineOperand<T> op{};
    op.base = buf(s.base); op.base_j = s.base_j;
    op.src = buf(s.src); op.src_j = s.src_j; op.src_ds = s.src_ds; op.cpl = s.cpl; op.neg = s.neg;
    op.out = buf(s.out); op.out_j = s.out_j; op.out_mode = s.out_mode;
    op.acc = buf(s.acc); op.acc_j = s.acc_j; op.acc_mode = s.acc_mode;
    op.s0 = s.s0; op.ns = s.ns; op.N = E.N; op.C = C;
    const T* A = Fb + (size_t)s.f * blk;
    const int ncols = s.ns * C;
    if (ncols <= 8 && partial_buf && partial_bytes >= (size_t)E.m * ncols * sizeof(T) &&
        (size_t)E.m * ncols * sizeof(T) <= gemv_cap) {
      T* xs = reinterpret_cast<T*>(partial_buf);  // narrow steps leave the split-K buffer free
      line_xbuild_kernel<R><<<E.grid_for((size_t)E.m * ncols), 256, 0, E.stream>>>(E.m, op, E.coef, xs);
      constexpr int RPC = 4;
      line_gemv_split_kernel<R, RPC><<<(E.m + RPC - 1) / RPC, 256, 0, E.stream>>>(A, E.ldf, E.m, op, xs);
      E.count_launch(2);
    } else if (ncols <= 8 && (size_t)E.m * ncols * sizeof(T) <= gemv_cap) {
      line_gemv_kernel<R><<<(E.m + 7) / 8, 256, (size_t)E.m * ncols * sizeof(T), E.stream>>>(A, E.ldf, E.m, op,
                                                                                          E.coef);
      E.count_launch();
    } else if (std::is_same<R, float>::value && E.tc_ready && C % 2 == 0) {
      LineOperand<float2> opf;
      std::memcpy(&opf, &op, sizeof(opf));
      const auto it = E.tc_tuned.find(C);
      const Engine::TcChoice ch = it != E.tc_tuned.end() ? it->second : Engine::TcChoice{};
      if (tick_gemm) E.tick_begin(Engine::K_GEMM);
      const cudaError_t le = launch_tc_shape(E, ch.shape, opf, s.f, C, ch.nsplit, Rin, partial_buf, partial_bytes,
                                             ch.cluster);
      if (le != cudaSuccess) return le;
      if (tick_gemm) E.tick_end(Engine::K_GEMM, step_bytes(E, s, C), 8.0 * E.m * E.m * (double)ncols);
    } else {
      const int gx = (E.m + BM - 1) / BM, gy = (ncols + BN - 1) / BN;
      // split K until about two CTAs per SM are busy (each slice at least two K tiles)
      int nsplit = std::max(1, std::min(8, (2 * E.num_sms + gx * gy - 1) / (gx * gy)));
      while (nsplit > 1 && (E.m + nsplit - 1) / nsplit < 2 * BK) --nsplit;
      while (nsplit > 1 && (size_t)nsplit * E.m * ncols * sizeof(T) > partial_bytes) --nsplit;
      const int kchunk = ((E.m + nsplit - 1) / nsplit + BK - 1) / BK * BK;
      T* partial = nsplit > 1 ? reinterpret_cast<T*>(partial_buf) : nullptr;
      if (tick_gemm) E.tick_begin(Engine::K_GEMM);
      gemm_fn<<<dim3(gx, gy, nsplit), 256, gemm_smem, E.stream>>>(A, E.ldf, E.m, op, E.coef, kchunk, partial);
      E.count_launch();
      if (nsplit > 1) {
        split_reduce_kernel<R><<<E.grid_for((size_t)E.m * ncols), 256, 0, E.stream>>>(partial, nsplit, E.m, op);
        E.count_launch();
      }
      if (tick_gemm) E.tick_end(Engine::K_GEMM, step_bytes(E, s, C), 8.0 * E.m * E.m * (double)ncols);
    }
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_group_simt(Engine& E, const SweepPhase& ph, const GArrays& arrs, int C, void* partial_buf,
                              size_t partial_bytes);
template <typename R>
cudaError_t launch_copy_phase(Engine& E, const SweepPhase& ph, const GArrays& arrs, int C);
cudaError_t launch_tc_group(Engine& E, int shape, const SweepPhase& ph, const GArrays& arrs, int C);

// Algorithmic work of a grouped step: every task reads its terms' blocks and input lines once,
// writes its output line (and reads its base, or the output itself when it adds to it).
static double group_bytes(const Engine& E, const SweepPhase& ph, int C) {
  const double e = (double)E.sweep_elem(), blkb = (double)E.m * E.m * e;
  double b = 0;
  for (const GTask& t : ph.tasks) {
    const double line = (double)E.m * t.ns * C * e;
    b += t.nterm * (blkb + line) + line * (1 + (t.base_arr != SB_NONE || t.mode == OUT_ADD));
    for (int q = 0; q < t.nterm; ++q) b += t.term[q].barr ? line : 0.0;  // a term's own base line
  }
  return b;
}
static double group_flops(const Engine& E, const SweepPhase& ph, int C) {
  double f = 0;
  for (const GTask& t : ph.tasks) f += 8.0 * E.m * E.m * (double)t.ns * C * t.nterm;
  return f;
}

// The phases of a sweep program in order: runs of block-Thomas steps, grouped steps (on the
// tensor cores for complex64 with an even column count) and line copies.
int run_persistent(Engine& E, const GArrays& arrs, int C, bool single, void* partial_buf, size_t partial_bytes);
int prepare_persistent(Engine& E, int C, size_t partial_bytes);

int run_lowp(Engine& E, const GArrays& arrs, int C, bool single);

template <typename R>
static cudaError_t launch_steps_t(Engine& E, const GArrays& arrs, int C, bool single, void* partial_buf,
                                  size_t partial_bytes, bool allow_tick) {
  if (std::is_same<R, float>::value && E.lowp) {
    const int lrc = run_lowp(E, arrs, C, single);
    if (lrc == HH_OK) return cudaSuccess;
    if (lrc != HH_EINVAL) return cudaErrorLaunchFailure;
  }
  if (std::is_same<R, float>::value && E.opts.persistent) {
    const int prc = run_persistent(E, arrs, C, single, partial_buf, partial_bytes);
    if (prc == HH_OK) return cudaSuccess;
    if (prc != HH_EINVAL) return cudaErrorLaunchFailure;
  }
  const std::vector<SweepPhase>& prog = E.program(C, single);
  const bool tick_gemm = allow_tick && E.opts.profile;
  for (size_t pi = 0; pi < prog.size();) {
    const SweepPhase& ph = prog[pi];
    if (ph.kind == PH_STEP) {
      std::vector<SweepStep> run;
      while (pi < prog.size() && prog[pi].kind == PH_STEP) run.push_back(prog[pi++].step);
      const cudaError_t ce = run_steps_t<R>(E, run, arrs, C, partial_buf, partial_bytes, allow_tick);
      if (ce != cudaSuccess) return ce;
      continue;
    }
    cudaError_t ce;
    if (ph.kind == PH_COPY) {
      ce = launch_copy_phase<R>(E, ph, arrs, C);
    } else if (std::is_same<R, float>::value && E.tc_ready && C % 2 == 0) {
      const auto it = E.tc_tuned.find(C);
      const int shape = it != E.tc_tuned.end() ? it->second.shape : 0;
      if (tick_gemm) E.tick_begin(Engine::K_GEMM);
      ce = launch_tc_group(E, shape, ph, arrs, C);
      if (tick_gemm) E.tick_end(Engine::K_GEMM, group_bytes(E, ph, C), group_flops(E, ph, C));
    } else {
      ce = launch_group_simt<R>(E, ph, arrs, C, partial_buf, partial_bytes);
    }
    if (ce != cudaSuccess) return ce;
    ++pi;
  }
  return cudaGetLastError();
}

double Engine::sweep_flops(int C, bool single) const {
  const std::vector<SweepPhase>& prog = program(C, single);
  double f = 0;
  for (const SweepPhase& p : prog) {
    if (p.kind == PH_STEP) f += 8.0 * m * m * (double)p.step.ns * C;
    else if (p.kind == PH_GROUP) f += group_flops(*this, p, C);
  }
  return f;
}

double Engine::sweep_bytes(int C, bool single) const {
  const std::vector<SweepPhase>& prog = program(C, single);
  double b = 0;
  for (const SweepPhase& p : prog) {
    if (p.kind == PH_STEP) b += step_bytes(*this, p.step, C);
    else if (p.kind == PH_GROUP) b += group_bytes(*this, p, C);
    else b += 2.0 * m * p.tasks[0].ns * C * sweep_elem();
  }
  return b;
}

int Engine::run_sweep(const void* Rin, void* V, void* W, int C, bool single) {
  tick_begin(K_SWEEP);
  const int rc = run_sweep_untimed(Rin, V, W, C, single, w_partial, w_partial_bytes);
  tick_end(K_SWEEP, sweep_bytes(C, single), sweep_flops(C, single));
  last_columns = C;
  return rc;
}

int Engine::run_sweep_untimed(const void* Rin, void* V, void* W, int C, bool single, void* partial,
                              size_t partial_bytes, bool allow_graph, void* T0, void* T1) {
  // Every sample_every()-th sweep of a profiled handle, and the sweep of every timed Arnoldi step, times
  // its GEMM steps one by one and so runs eagerly; the others replay a captured graph.
  if (precision == HH_PREC_FP32 && tc_ready && allow_graph && C % 2 == 0 && !tc_tuned.count(C)) {
    const int rc = tune_tc(C, Rin, V, W, partial, partial_bytes);
    if (rc) return rc;
  }
  if ((opts.bcr_depth < 0 || (opts.twisted < 0 && twisted_ok(C))) && allow_graph && !bcr_tuned.count(C)) {
    const int rc = tune_depth(C, Rin, V, W, partial, partial_bytes);
    if (rc) return rc;
  }
  if (allow_graph) {
    const int rc = prepare_persistent(*this, C, partial_bytes);
    if (rc) return rc;
  }
  const bool sampled = opts.profile && ((sweep_calls++ % sample_every() == 0) || sample_next_sweep);
  sample_next_sweep = false;
  GArrays arrs{};
  arrs.p[SB_RIN] = const_cast<void*>(Rin);
  arrs.p[SB_V] = V;
  arrs.p[SB_W] = W;
  arrs.p[SB_T0] = T0 ? T0 : w_t0;
  arrs.p[SB_T1] = T1 ? T1 : w_t1;
  auto launch = [&](bool tick) {
    return precision == HH_PREC_FP32 ? launch_steps_t<float>(*this, arrs, C, single, partial, partial_bytes, tick)
                                     : launch_steps_t<double>(*this, arrs, C, single, partial, partial_bytes, tick);
  };
  if (!opts.use_graph || !allow_graph || sampled) {
    cudaError_t ce = launch(sampled);
    if (ce != cudaSuccess) { set_cuda_error(ce, "sweep launch"); return HH_ECUDA; }
    return HH_OK;
  }
  cudaGraphExec_t exec = nullptr;
  int64_t per_replay = 0;
  for (const SweepGraph& g : sweep_graphs)
    if (g.rin == Rin && g.v == V && g.w == W && g.partial == partial && g.C == C && g.single == single) {
      exec = g.exec;
      per_replay = g.kernels;
    }
  if (!exec) {
    cudaGraph_t graph = nullptr;
    const int64_t before = kernel_launches;
    cudaError_t ce = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      const cudaError_t le = launch(false);
      ce = cudaStreamEndCapture(stream, &graph);
      if (ce == cudaSuccess) ce = le;
    }
    per_replay = kernel_launches - before;
    kernel_launches = before;  // counted at every replay instead
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      set_cuda_error(ce, "sweep graph capture");
      return HH_ECUDA;
    }
    sweep_graphs.push_back(SweepGraph{Rin, V, W, partial, C, single, exec, per_replay});
  }
  cudaError_t ce = cudaGraphLaunch(exec, stream);
  if (ce != cudaSuccess) { set_cuda_error(ce, "sweep graph launch"); return HH_ECUDA; }
  count_launch((int)per_replay);
  return HH_OK;
}

int Engine::sweep_inline(const void* Rin, void* V, void* W, int C, bool single) {
  GArrays arrs{};
  arrs.p[SB_RIN] = const_cast<void*>(Rin);
  arrs.p[SB_V] = V;
  arrs.p[SB_W] = W;
  arrs.p[SB_T0] = w_t0;
  arrs.p[SB_T1] = w_t1;
  cudaError_t ce = precision == HH_PREC_FP32
                       ? launch_steps_t<float>(*this, arrs, C, single, w_partial, w_partial_bytes, false)
                       : launch_steps_t<double>(*this, arrs, C, single, w_partial, w_partial_bytes, false);
  if (ce != cudaSuccess) { set_cuda_error(ce, "sweep launch"); return HH_ECUDA; }
  return HH_OK;
}

int Engine::ensure_tuned(int C) {
  if (precision == HH_PREC_FP32 && tc_ready && C % 2 == 0 && !tc_tuned.count(C)) {
    const int rc = tune_tc(C, w_rin, w_v, w_w, w_partial, w_partial_bytes);
    if (rc) return rc;
  }
  if ((opts.bcr_depth < 0 || (opts.twisted < 0 && twisted_ok(C))) && !bcr_tuned.count(C)) {
    const int rc = tune_depth(C, w_rin, w_v, w_w, w_partial, w_partial_bytes);
    if (rc) return rc;
  }
  return prepare_persistent(*this, C, w_partial_bytes);
}

// Autotuner of the strip-solve form for C columns per strip: block Thomas, every cyclic-reduction
// depth whose blocks are stored and the twisted factorisation (when it can run C columns) run
// whole sweeps (one warm-up, three timed with CUDA events, on the arrays of the call, whose
// outputs the real sweep overwrites next) and the fastest is kept.
int Engine::tune_depth(int C, const void* Rin, void* V, void* W, void* partial, size_t partial_bytes) {
  std::vector<int> cand = {0};
  for (int d = 1; d <= bdir.dmax; ++d)
    if (bdir.iDeep[d] >= 0) cand.push_back(d);
  if (twisted_ok(C)) cand.push_back(PROG_TWISTED);
  if (cand.size() == 1) {
    bcr_tuned[C] = 0;
    return HH_OK;
  }
  GArrays arrs{};
  arrs.p[SB_RIN] = const_cast<void*>(Rin);
  arrs.p[SB_V] = V;
  arrs.p[SB_W] = W;
  arrs.p[SB_T0] = w_t0;
  arrs.p[SB_T1] = w_t1;
  const bool single = opts.single_sweep != 0;
  auto sweep = [&]() {
    return precision == HH_PREC_FP32 ? launch_steps_t<float>(*this, arrs, C, single, partial, partial_bytes, false)
                                     : launch_steps_t<double>(*this, arrs, C, single, partial, partial_bytes, false);
  };
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  int best = 0;
  float best_ms = 1e30f;
  for (int d : cand) {
    bcr_tuned[C] = d;
    if (sweep() != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaEventRecord(a, stream);
    for (int r = 0; r < 3; ++r) sweep();
    cudaEventRecord(b, stream);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best_ms) {
      best_ms = ms;
      best = d;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  bcr_tuned[C] = best;
  return check_device_error("cyclic-reduction depth autotune");
}

// launch helpers used by krylov.cu / api.cu / noalloc.cu
template <typename R>
static void launch_pack_t(Engine& E, const double2* const* srcptr, const double* scale, int C, int t, int4 codes,
                          void* X) {
  pack_kernel<R><<<E.grid_for(E.sweep_ws_bytes(C) / E.sweep_elem()), 256, 0, E.stream>>>(
      srcptr, scale, C, t, codes, E.n, E.N, E.R, reinterpret_cast<typename Cx<R>::T*>(X));
  E.count_launch();
}
template <typename R>
static void launch_unpack_t(Engine& E, const void* X, int C, int t, int4 codes, double2* dst, size_t stride) {
  unpack_kernel<R><<<E.grid_for(E.sweep_ws_bytes(C) / E.sweep_elem()), 256, 0, E.stream>>>(
      reinterpret_cast<const typename Cx<R>::T*>(X), C, t, codes, E.n, E.N, E.R, dst, stride);
  E.count_launch();
}

void launch_pack(Engine& E, const double2* const* srcptr, const double* scale, int C, int t, int4 codes, void* X) {
  if (E.precision == HH_PREC_FP32) launch_pack_t<float>(E, srcptr, scale, C, t, codes, X);
  else launch_pack_t<double>(E, srcptr, scale, C, t, codes, X);
}
void launch_unpack_tab(Engine& E, const void* X, int C, int t, int4 codes, double2* const* dstcol) {
  if (E.precision == HH_PREC_FP32)
    unpack_tab_kernel<float><<<E.grid_for(E.sweep_ws_bytes(C) / E.sweep_elem()), 256, 0, E.stream>>>(
        reinterpret_cast<const float2*>(X), C, t, codes, E.n, E.N, E.R, dstcol);
  else
    unpack_tab_kernel<double><<<E.grid_for(E.sweep_ws_bytes(C) / E.sweep_elem()), 256, 0, E.stream>>>(
        reinterpret_cast<const double2*>(X), C, t, codes, E.n, E.N, E.R, dstcol);
  E.count_launch();
}
// hi = F rounded to TF32, lo = F - hi, elementwise over the whole complex64 factor store
__global__ void tf32_split_kernel(const float* __restrict__ F, float* __restrict__ hi, float* __restrict__ lo,
                                  size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    float h, l;
    tc::split_tf32(F[i], h, l);
    hi[i] = h;
    lo[i] = l;
  }
}

void set_tc_group_attributes();
void set_persist_attributes();
void set_lowp_attributes();

int Engine::load_encoder() {
  if (precision != HH_PREC_FP32 || !opts.tensor_cores) return HH_OK;
  if (encode_fn) return HH_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return HH_ECUDA;
  }
  encode_fn = fn;
  cudaFuncSetAttribute((const void*)tc_line_gemm_kernel<tc::Wide>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::Wide::SMEM);
  cudaFuncSetAttribute((const void*)tc_line_gemm_kernel<tc::Narrow>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::Narrow::SMEM);
  cudaFuncSetAttribute((const void*)tc_line_gemm_kernel<tc::Wide, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::Wide::SMEM);
  cudaFuncSetAttribute((const void*)tc_line_gemm_kernel<tc::Narrow, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::Narrow::SMEM);
  cudaFuncSetAttribute((const void*)tc_line_gemm_kernel<tc::Huge>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::Huge::SMEM);
  cudaFuncSetAttribute((const void*)tc_line_gemm_kernel<tc::Huge, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::Huge::SMEM);
  set_tc_group_attributes();
  set_persist_attributes();
  set_lowp_attributes();
  return HH_OK;
}

void Engine::free_dense_scratch() {
  dfree(dense_hi);
  dfree(dense_lo);
  dense_hi = dense_lo = nullptr;
  for (DenseMaps& d : dense_maps) d.ptr = nullptr;
}

// Rows [r0, m) of C = (+/-) A B (+ C), on the CUDA cores in FP32: the few rows below the last
// full 128-row tile, so that the tensor-core grid fits in one wave (at m = 1025 a full grid
// is 9 x 17 = 153 CTAs of one per SM: the 153rd would run alone).  A is read as hi + lo (its
// exact split), since C may be A itself.  Grid (columns / 32, rows); 32 warps split K.  It
// lets the tensor-core kernel (launched next, with programmatic dependent launch) start at
// once: the two run side by side, on disjoint rows of C.
__global__ void __launch_bounds__(1024) dense_tail_rows_kernel(const float2* __restrict__ Ahi,
                                                               const float2* __restrict__ Alo,
                                                               const float2* __restrict__ B, float2* Cm, int ld,
                                                               int m, int r0, int neg, int add) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ float2 part[32][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane, r = r0 + blockIdx.y;
  float2 acc = make_float2(0.f, 0.f);
  if (c < m) {
#pragma unroll 4
    for (int k = w; k < m; k += 32) {
      const float2 h = Ahi[(size_t)r * ld + k], l = Alo[(size_t)r * ld + k];
      cfma(acc, make_float2(h.x + l.x, h.y + l.y), B[(size_t)k * ld + c]);
    }
  }
  part[w][lane] = acc;
  __syncthreads();
  if (w == 0 && c < m) {
    float2 z = part[0][lane];
#pragma unroll
    for (int q = 1; q < 32; ++q) z = cadd(z, part[q][lane]);
    if (neg) z = make_float2(-z.x, -z.y);
    float2* o = Cm + (size_t)r * ld + c;
    *o = add ? cadd(*o, z) : z;
  }
}

int Engine::tc_dense_gemm(const void* A, const void* B, void* C, bool negate_b, bool add) {
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(encode_fn);
  if (!encode) return (set_error("tensor-map encoder not loaded"), HH_ECUDA);
  const cuuint64_t dims[3] = {(cuuint64_t)2 * m, (cuuint64_t)m, 1};
  const cuuint64_t strides[2] = {(cuuint64_t)ldf * 2 * sizeof(float), (cuuint64_t)m * ldf * 2 * sizeof(float)};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (!dense_hi) {
    const size_t bytes = (size_t)m * ldf * 2 * sizeof(float);
    if (dmalloc(&dense_hi, bytes) || dmalloc(&dense_lo, bytes)) return HH_ENOMEM;
    const cuuint32_t box[3] = {32, (cuuint32_t)tc::BM, 1};
    for (int h = 0; h < 2; ++h)
      if (encode(h ? &dense_map_lo : &dense_map_hi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h ? dense_lo : dense_hi, dims,
                 strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return (set_error("cuTensorMapEncodeTiled failed for the setup scratch"), HH_ECUDA);
  }
  // B viewed as rows of 2 ldf floats (the line operand of the step kernel, one line)
  DenseMaps* dm = nullptr;
  for (DenseMaps& d : dense_maps)
    if (d.ptr == B) dm = &d;
  if (!dm) {
    dm = &dense_maps[dense_maps_next];
    dense_maps_next = (dense_maps_next + 1) % 4;
    const cuuint64_t bd[3] = {(cuuint64_t)2 * ldf, (cuuint64_t)m, 1};
    const cuuint32_t box_b[3] = {(cuuint32_t)(2 * tc::Wide::BNC), (cuuint32_t)tc::RAW_BASE_ROWS, 1};
    const cuuint32_t box_s[3] = {(cuuint32_t)(2 * tc::Wide::BNC), (cuuint32_t)tc::RAW_SRC_ROWS, 1};
    void* p = const_cast<void*>(B);
    if (encode(&dm->base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p, bd, strides, box_b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        encode(&dm->src, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p, bd, strides, box_s, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      dm->ptr = nullptr;
      return (set_error("cuTensorMapEncodeTiled failed for a setup matrix"), HH_ECUDA);
    }
    dm->ptr = B;
  }
  const size_t nfloat = (size_t)m * ldf * 2;
  tf32_split_kernel<<<grid_for(nfloat), 256, 0, stream>>>(reinterpret_cast<const float*>(A),
                                                         reinterpret_cast<float*>(dense_hi),
                                                         reinterpret_cast<float*>(dense_lo), nfloat);
  LineOperand<float2> op{};
  if (negate_b) {  // x = 0 - identity(B)
    op.src = reinterpret_cast<const float2*>(B);
    op.cpl = XC_IDENT;
    op.neg = 1;
  } else {
    op.base = reinterpret_cast<const float2*>(B);
    op.cpl = XC_NONE;
  }
  op.out = reinterpret_cast<float2*>(C);
  op.out_mode = add ? OUT_ADD : OUT_SET;
  op.s0 = 0; op.ns = m; op.N = ldf; op.C = 1;  // a node row = one row of the matrix
  const int gx = (m + tc::BM - 1) / tc::BM, gy = (m + tc::Wide::BNC - 1) / tc::Wide::BNC;
  const int kchunk = (m + tc::BKC - 1) / tc::BKC * tc::BKC;
  // one CTA per SM: when the grid is just over one wave, the last few rows go to the CUDA cores
  const int full = m / tc::BM, tail = m - full * tc::BM;
  const bool split_tail = gx * gy > num_sms && full >= 1 && tail > 0 && tail <= 8 && full * gy <= num_sms;
  if (split_tail) {
    dense_tail_rows_kernel<<<dim3((m + 31) / 32, tail), 1024, 0, stream>>>(
        reinterpret_cast<const float2*>(dense_hi), reinterpret_cast<const float2*>(dense_lo),
        reinterpret_cast<const float2*>(B), reinterpret_cast<float2*>(C), ldf, m, full * tc::BM, negate_b ? 1 : 0,
        add ? 1 : 0);
    count_launch();
  }
  // after the tail kernel: programmatic dependent launch, so that the two overlap (the
  // tensor-core kernel waits for it only before writing its output)
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(split_tail ? full : gx, gy, 1);
  cfg.blockDim = dim3(tc::THREADS);
  cfg.dynamicSmemBytes = tc::Wide::SMEM;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = split_tail ? 1 : 0;
  float2* nopartial = nullptr;
  const cudaError_t ce = cudaLaunchKernelEx(&cfg, tc_line_gemm_kernel<tc::Wide, false>, dense_map_hi, dense_map_lo,
                                            dm->base, dm->src, 0, m, op, coef, kchunk, nopartial, err,
                                            opts.timeout_cycles);
  count_launch(2);
  if (ce != cudaSuccess) return (set_cuda_error(ce, "tensor-core setup GEMM launch"), HH_ECUDA);
  return HH_OK;
}

int Engine::prepare_tensor_cores() {
  if (precision != HH_PREC_FP32 || !opts.tensor_cores) return HH_OK;
  int rc = load_encoder();
  if (rc) return rc;
  free_dense_scratch();
  const size_t nfloat = (size_t)factor_blocks() * m * ldf * 2;
  if (dmalloc(&factors_hi, nfloat * sizeof(float)) || dmalloc(&factors_lo, nfloat * sizeof(float))) return HH_ENOMEM;
  tf32_split_kernel<<<grid_for(nfloat), 256, 0, stream>>>(reinterpret_cast<const float*>(factors),
                                                         reinterpret_cast<float*>(factors_hi),
                                                         reinterpret_cast<float*>(factors_lo), nfloat);
  count_launch();
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(encode_fn);
  // rows of 2m floats (interleaved complex), m rows per block, factor_blocks() blocks
  const cuuint64_t dims[3] = {(cuuint64_t)2 * m, (cuuint64_t)m, (cuuint64_t)factor_blocks()};
  const cuuint64_t strides[2] = {(cuuint64_t)ldf * 2 * sizeof(float), (cuuint64_t)m * ldf * 2 * sizeof(float)};
  const cuuint32_t box[3] = {32, (cuuint32_t)tc::BM, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int h = 0; h < 3; ++h) {
    CUtensorMap* mp = h == 2 ? &tmap_c : (h ? &tmap_lo : &tmap_hi);
    void* src = h == 2 ? factors : (h ? factors_lo : factors_hi);
    CUresult r = encode(mp, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, src, dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
      return HH_ECUDA;
    }
  }
  tc_ready = true;
  return HH_OK;
}

// Autotuner of the tensor-core step for C columns per strip: one representative wide step
// (all strips, coupled operand) is timed with CUDA events for each tile shape and K split
// (one warm-up and three timed launches each, writing to a scratch array), and the fastest
// is kept for every later sweep with this column count.
// the autotuner's candidates: K splits summed by split_reduce_kernel (0 = fill the SMs), then
// K splits summed in a thread-block cluster
static const int kTcSplits[7] = {0, 1, 2, 4, 2, 4, 8};
static bool tc_candidate_cluster(int variant) { return variant >= 4; }

int Engine::tune_tc(int C, const void* Rin, void* V, void* W, void* partial, size_t partial_bytes) {
  if (opts.autotune == 0) {
    tc_tuned[C] = TcChoice{};
    return HH_OK;
  }
  if (opts.autotune < 0) {  // one candidate, chosen by the caller: -(1 + 7 shape + variant)
    const int idx = -opts.autotune - 1;
    const int variant = idx % 7;
    tc_tuned[C] = TcChoice{(idx / 7) % kTcShapes, kTcSplits[variant], tc_candidate_cluster(variant), 0.0};
    return HH_OK;
  }
  const std::vector<SweepStep>& steps = opts.single_sweep ? steps_single : steps_double;
  const SweepStep* pick = nullptr;
  for (const SweepStep& s : steps)
    if (s.ns == N && s.src != SB_NONE && (!pick || s.cpl > pick->cpl)) pick = &s;
  if (!pick) {
    tc_tuned[C] = TcChoice{};
    return HH_OK;
  }
  void* tmp = nullptr;
  if (dmalloc(&tmp, sweep_ws_bytes(C))) return HH_ENOMEM;
  auto buf = [&](int b) -> float2* {
    return b == SB_RIN ? (float2*)Rin : (b == SB_V ? (float2*)V : (b == SB_W ? (float2*)W : nullptr));
  };
  LineOperand<float2> op{};
  op.base = buf(pick->base); op.base_j = pick->base_j;
  op.src = buf(pick->src); op.src_j = pick->src_j; op.src_ds = pick->src_ds; op.cpl = pick->cpl; op.neg = pick->neg;
  op.out = (float2*)tmp; op.out_j = pick->out_j; op.out_mode = OUT_SET;
  op.acc = nullptr; op.acc_j = 0; op.acc_mode = 0;
  op.s0 = pick->s0; op.ns = pick->ns; op.N = N; op.C = C;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  auto elapsed_us = [&]() {
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    return (double)ms * 1e3;
  };
  // stage 1: every candidate on the representative step, repeated (its factor block stays in
  // L2 after the first run)
  std::vector<TcChoice> ranked;
  for (int shape = 0; shape < kTcShapes; ++shape)
    for (int variant = 0; variant < 7; ++variant) {
      const bool cl = tc_candidate_cluster(variant);
      const int ns = kTcSplits[variant];
      auto run = [&]() { return launch_tc_shape(*this, shape, op, pick->f, C, ns, Rin, partial, partial_bytes, cl); };
      if (run() != cudaSuccess) {  // e.g. a cluster shape the GPU cannot co-schedule
        cudaGetLastError();
        continue;
      }
      cudaEventRecord(a, stream);
      for (int r = 0; r < 3; ++r) run();
      cudaEventRecord(b, stream);
      ranked.push_back(TcChoice{shape, ns, cl, elapsed_us() / 3});
    }
  std::sort(ranked.begin(), ranked.end(), [](const TcChoice& x, const TcChoice& y) { return x.us < y.us; });
  // stage 2: the three best on a run of consecutive steps over different factor blocks, as in
  // a sweep (each block read from HBM, each step overlapping the previous one's end)
  TcChoice best;
  best.us = 1e30;
  const int nf = std::min(16, R + 1);
  for (size_t q = 0; q < ranked.size() && q < 3; ++q) {
    const TcChoice& c = ranked[q];
    auto seq = [&]() {
      for (int f = 0; f < nf; ++f) launch_tc_shape(*this, c.shape, op, f, C, c.nsplit, Rin, partial, partial_bytes, c.cluster);
    };
    seq();
    cudaEventRecord(a, stream);
    for (int r = 0; r < 2; ++r) seq();
    cudaEventRecord(b, stream);
    const double us = elapsed_us() / (2 * nf);
    if (us < best.us) best = TcChoice{c.shape, c.nsplit, c.cluster, us};
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaStreamSynchronize(stream);
  dfree(tmp);
  tc_tuned[C] = best;
  return check_device_error("tensor-core autotune");
}

const Engine::LineMaps* Engine::line_maps_for(const void* buf, int C, int bnc, int lines) {
  if (lines <= 0) lines = R + 1;
  for (const LineMaps& lm : line_maps)
    if (lm.ptr == buf && lm.C == C && lm.bnc == bnc && lm.lines == lines) return &lm;
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(encode_fn);
  if (!encode || C % 2) return nullptr;
  LineMaps& lm = line_maps[line_maps_next];
  line_maps_next = (line_maps_next + 1) % 24;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * N * C, (cuuint64_t)m, (cuuint64_t)lines};
  const cuuint64_t strides[2] = {(cuuint64_t)2 * N * C * sizeof(float), (cuuint64_t)m * 2 * N * C * sizeof(float)};
  const cuuint32_t estr[3] = {1, 1, 1};
  const cuuint32_t box_b[3] = {(cuuint32_t)(2 * bnc), (cuuint32_t)tc::RAW_BASE_ROWS, 1};
  const cuuint32_t box_s[3] = {(cuuint32_t)(2 * bnc), (cuuint32_t)tc::RAW_SRC_ROWS, 1};
  void* p = const_cast<void*>(buf);
  if (encode(&lm.base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p, dims, strides, box_b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      encode(&lm.src, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p, dims, strides, box_s, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
    lm.ptr = nullptr;
    set_error("cuTensorMapEncodeTiled failed for a sweep array");
    return nullptr;
  }
  lm.ptr = buf;
  lm.C = C;
  lm.bnc = bnc;
  lm.lines = lines;
  return &lm;
}

void launch_unpack(Engine& E, const void* X, int C, int t, int4 codes, double2* dst, size_t stride) {
  if (E.precision == HH_PREC_FP32) launch_unpack_t<float>(E, X, C, t, codes, dst, stride);
  else launch_unpack_t<double>(E, X, C, t, codes, dst, stride);
}

}  // namespace hh
