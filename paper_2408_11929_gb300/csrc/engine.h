// Host-side engine: one per hh_handle.  Owns the device, stream, strip factors and the
// Krylov slots; the kernels live in setup.cu, sweep.cu and krylov.cu.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hh.h"
#include "common.cuh"

namespace hh {

void set_error(const std::string& msg);
struct Engine;
// H = V^H W and W <- W - V H (one block classical Gram-Schmidt pass, krylov.cu)
int gram_schmidt_pass(Engine& E, int p, const double2* V, int t, double2* W, double2* H_host);

// One step of the batched sweep (see sweep.cu): for strips s0 .. s0+ns-1,
//   out[out_j] (set / -= / +=) F_f * x,   x = base[base_j] +- C(src[src_j], strip s + src_ds)
// with C the identity or the coupling to the line below (L) / above (U), and optionally the
// result also accumulated into acc[acc_j].  Buffers: SB_RIN (packed right-hand sides), SB_V
// (sweep result), SB_W (corrections).
enum SweepBuf { SB_NONE = 0, SB_RIN = 1, SB_V = 2, SB_W = 3, SB_T0 = 4, SB_T1 = 5, SB_COUNT = 6 };
struct SweepStep {
  int f, s0, ns;
  int base, base_j;
  int src, src_j, src_ds, cpl, neg;
  int out, out_j, out_mode;
  int acc, acc_j, acc_mode;
};

std::vector<SweepStep> build_steps(int n, int N, bool double_sweep);

// A grouped step (sweep.cu, group.cu): independent output lines ("tasks"), each
//   out[out_line] = (base[base_line] or, with OUT_ADD, out itself, else 0) + sum_q (-1)^neg_q F_{f_q} x_q
// over strips s0 .. s0+ns-1, x_q = line `line` of array `arr` (a SweepBuf) at strip s + ds
// (zero outside 0..N-1).  The terms' K ranges are concatenated.  T0 and T1 hold one line.
struct GTerm {
  int f, arr, line, ds, neg;
  // optional: x = xbase[bline] + (-1)^neg C(arr[line]), C the identity (cpl = XC_NONE) or the
  // coupling to the node line below / above (XC_LOWER / XC_UPPER), as in a block-Thomas step
  int cpl = 0, barr = 0, bline = 0;
};
constexpr int GMAX_TERMS = 3;
struct GTask {
  int nterm;
  GTerm term[GMAX_TERMS];
  int out_arr, out_line, base_arr, base_line, mode, s0, ns;
};
// One phase of a sweep program: a step of the line-coupled block-Thomas form, a grouped step,
// or a copy of one line (strips s0 .. s0+ns-1) from task 0's term 0 line to its output line.
enum PhaseKind { PH_STEP = 0, PH_GROUP = 1, PH_COPY = 2 };
struct SweepPhase {
  int kind;
  SweepStep step;
  std::vector<GTask> tasks;
  size_t dev_off = 0;  // first task in the engine's device task table
};
// Device addresses of the sweep arrays, by SweepBuf.  Rin, V, W hold R+1 lines, T0 and T1 one.
struct GArrays {
  void* p[SB_COUNT];
};
// Block directory of the factor store beyond F_0..F_R, G, K (see setup.cu).
struct BlockDir {
  int iY = -1;   // D_int^{-1}[j, 0] L, j = 0..R-1 (strips visited before the last)
  int iYL = -1;  // D_last^{-1}[j, 0] L, j = 0..R (the last strip)
  int iZ = -1;   // D_int^{-1}[j, R-1] U, j = 1..R-1 at iZ + j - 1
  int iGp = -1;  // G^(2^l), l = 1..LF-1 at iGp + l - 1
  int iKp = -1;  // K^(2^l), l = 1..LB-1 at iKp + l - 1
  int LF = 0, LB = 0;  // levels of the forward / backward interface scans
  // block cyclic reduction of the strip solves (levels 1..dmax): at level l the odd lines of
  // the level-(l-1) system are eliminated; its blocks are Dinv = D_int^{-1}, L Dinv, U Dinv,
  // Dinv L, Dinv U at iLev + 5 (l - 1) + 0..4.  For each depth d in 1..dmax the block-Thomas
  // factors of the reduced system (nd = R / 2^d lines, the last strip one more): F_0..F_{nd-1},
  // F_top, G_1..G_{nd-1} (F_i L), G_top, H_0..H_{nd-1} (F_i U) from iDeep[d].
  int dmax = 0, iLev = -1;
  int iDeep[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
  // twisted block factorisation of the strip solves (lines 0..R-1 of every strip, meeting at
  // line q = R/2): G_j = P_j^{-1} from the bottom, P_{R-1} = D_int, P_j = D_int - U G_{j+1} L
  // (j = R-1 .. q+1, at iTw + j - q - 1); M = (D_int - L F_{q-1} U - U G_{q+1} L)^{-1} at iTwM;
  // Z_0 = D_int^{-1}[0, R-1] U at iZ0 (the last strip's extra line enters through Z_0..Z_{R-1})
  int iTw = -1, iTwM = -1, iZ0 = -1, twq = 0;
  int total = 0;  // blocks in the store
};
// Index of the twisted program among the per-depth programs (0..7: cyclic-reduction depth).
constexpr int PROG_TWISTED = 8;
constexpr int NPROG = 9;
// form: interface form (0, 1); depths: bit d set = the blocks of cyclic-reduction depth d;
// twisted: the blocks of the twisted strip solves (form 1, N >= 2, R >= 4)
BlockDir block_directory(int R, int N, int form, unsigned depths = 0, bool twisted = false);
// depth: cyclic-reduction levels of the full-right-hand-side strip solves (0: block Thomas), or
// PROG_TWISTED for the twisted factorisation
std::vector<SweepPhase> build_program(int n, int N, bool double_sweep, int form, const BlockDir& bd, int depth = 0);
// whether the twisted strip solves can be stored for R lines per strip, N strips, form
bool twisted_possible(int R, int N, int form);
// largest usable depth: R divisible by 2^d (at most 7)
int max_bcr_depth(int R);

// Direction codes of the BT frame mapping (node of the BT frame -> node of the grid).
enum DirCode { DC_BT = 0, DC_TB = 1, DC_LR = 2, DC_RL = 3 };

class SlotSolver;  // continuous-batching MPGMRES driver (krylov.cu)
struct FdState;    // five-point finite differences with overlapping strips (fd.cu)
class Engine;
int fd_setup(Engine& E);
void fd_free(Engine& E);
int fd_precondition(Engine& E, const double2* const* src, const double* scale, int C, int t, int4 codes,
                    double2* const* dst, bool single);
void fd_operator(Engine& E, const double2* const* xcol, double2* const* ycol, int ncols);
void fd_load(Engine& E, const double* dsrc, int nsrc, double2* b);
int fd_reserve(Engine& E, int C);  // sweep buffers for C columns, before any graph capture
int fd_blocks(const Engine& E);     // stored m x m inverses

class Engine {
 public:
  // configuration
  int device = 0, num_sms = 0, coop_per_sm = 1;
  double k = 0;
  int n = 0, m = 0, N = 0, R = 0, ldf = 0;
  int precision = HH_PREC_FP64;
  std::vector<int> dir_codes;  // DirCode per preconditioner, in order LR, RL, BT, TB of the bits
  int t = 0;
  hh_opts opts{};
  Coef coef{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // hh_opts.discretization = HH_DISC_FD: the paper's five-point scheme and overlapping strips
  // (fd.cu); none of the P1 strip factors or sweep programs below exist then
  FdState* fd = nullptr;

  // device buffers
  void* factors = nullptr;  // R+3 blocks of m x ldf complex: F_0..F_R, G, K (setup.cu)
  // tensor-core operands (complex64 only): the factor store split into TF32 hi and lo
  // parts, and one 3-D tensor map over each (floats along a row, rows, blocks)
  void* factors_hi = nullptr;
  void* factors_lo = nullptr;
  CUtensorMap tmap_hi{}, tmap_lo{};
  CUtensorMap tmap_c{};  // the complex64 store itself, same view (persistent sweep kernel)
  bool tc_ready = false;
  int prepare_tensor_cores();  // sweep.cu
  // Dense complex64 GEMM C = A B (or A (-B)) of m x m blocks (leading dimension ldf) on the
  // tensor cores, for the setup: A is split into TF32 hi / lo scratch, B's rows are the
  // kernel's line operand.  load_encoder() must have succeeded.
  int load_encoder();
  bool tc_dense_ok() const { return encode_fn != nullptr; }
  int tc_dense_gemm(const void* A, const void* B, void* C, bool negate_b, bool add = false);
  void free_dense_scratch();
  void* dense_hi = nullptr;
  void* dense_lo = nullptr;
  CUtensorMap dense_map_hi{}, dense_map_lo{};
  struct DenseMaps {
    const void* ptr = nullptr;
    CUtensorMap base{}, src{};
  };
  DenseMaps dense_maps[4];
  int dense_maps_next = 0;
  // 3-D views of a sweep array (floats of a node row, node rows, lines) with the raw-row
  // boxes of the tensor-core step (16 and 18 rows), cached per (array, columns per strip)
  struct LineMaps {
    const void* ptr = nullptr;
    int C = -1, bnc = 0, lines = 0;
    CUtensorMap base{}, src{};
  };
  LineMaps line_maps[24];
  int line_maps_next = 0;
  void* encode_fn = nullptr;  // cuTensorMapEncodeTiled
  // lines: lines held by the array (0: R + 1, the sweep arrays; 1: the interface arrays)
  const LineMaps* line_maps_for(const void* buf, int C, int bnc, int lines = 0);
  // autotuned tensor-core step per column count: tile shape (0: 64 columns x 3 stages,
  // 1: 32 columns x 4 stages) and K split (0 = fill the SMs)
  struct TcChoice {
    int shape = 0, nsplit = 0;
    bool cluster = false;  // K slices summed in a thread-block cluster instead of split_reduce
    double us = 0;
  };
  std::map<int, TcChoice> tc_tuned;
  // clusters of the grouped tensor-core step that fit on the device at once, per (tile shape,
  // cluster size) (group.cu)
  std::map<int, int> group_clusters;
  int tune_tc(int C, const void* Rin, void* V, void* W, void* partial, size_t partial_bytes);
  // sweeps replayed as CUDA graphs (opts.use_graph), one per (arrays, columns, kind)
  struct SweepGraph {
    const void *rin, *v, *w, *partial;
    int C;
    bool single;
    cudaGraphExec_t exec;
    int64_t kernels;  // launches per replay
  };
  std::vector<SweepGraph> sweep_graphs;
  // grid barriers (GRID_BAR_WORDS words each): BAR_SETUP for the pivoted Gauss-Jordan of the
  // strip setup, BAR_CHAIN for the sweep's interface chains
  enum { BAR_SETUP = 0, BAR_CHAIN = 1, BAR_PERSIST = 2, BAR_COUNT = 3 };
  static constexpr size_t BAR_BYTES = (size_t)BAR_COUNT * 64 * sizeof(unsigned);
  unsigned* bar = nullptr;
  int* err = nullptr;       // device error word
  std::vector<SweepStep> steps_double, steps_single;  // sweep schedules (block-Thomas form)
  // sweep programs (opts.interface_form): phases of a double and of a single sweep, their
  // grouped tasks in one device table
  BlockDir bdir;
  // programs of every cyclic-reduction depth whose blocks are stored (index = depth) and of
  // the twisted strip solves (index PROG_TWISTED)
  std::vector<SweepPhase> prog_double_d[NPROG], prog_single_d[NPROG];
  int bcr_blocks();                          // setup.cu: the cyclic-reduction blocks of bdir
  std::map<int, int> bcr_tuned;              // program per column count (fixed or autotuned)
  int depth_for(int C) const;                // the program (depth or PROG_TWISTED) of C columns
  bool twisted_ok(int C) const;              // the twisted program can run C columns
  int twisted_blocks();                      // setup.cu: the twisted strip-solve blocks of bdir
  const std::vector<SweepPhase>& program(int C, bool single) const;
  int tune_depth(int C, const void* Rin, void* V, void* W, void* partial, size_t partial_bytes);
  GTask* prog_tasks = nullptr;
  int upload_programs();
  // the same programs for the persistent sweep kernel (persist.cu): block-Thomas steps as
  // grouped tasks, one device task table, device phase tables per (program, columns, shape)
  std::vector<SweepPhase> pprog_double_d[NPROG], pprog_single_d[NPROG];
  GTask* pprog_tasks = nullptr;
  std::map<int64_t, void*> pphase_cache;
  int upload_persistent();
  bool no_alloc_call = false;  // inside hh_apply_preconditioner_noalloc
  // device staging of host buffers passed to the C ABI (api.cu), grown on demand and kept
  std::recursive_mutex stage_mu;
  void* stage_buf[2] = {nullptr, nullptr};
  size_t stage_cap[2] = {0, 0};
  // HH_PREC_BF16 (lowp.cu): complex64 sweep lines and setup, bf16 factor store for the products
  bool lowp = false;
  void* factors_bf16 = nullptr;
  CUtensorMap tmap_bf16{};
  int prepare_lowp();
  size_t bytes_allocated = 0;

  // statistics
  // K_GEMM: the wide GEMM steps inside a sweep (GEMM launch + its split-K reduction), a subset
  // of K_SWEEP timed on their own
  // K_GSDOT: the Gram-Schmidt inner-product kernel alone (every launch), within K_GS
  enum KClass { K_SWEEP = 0, K_SPMV = 1, K_GS = 2, K_SETUP = 3, K_GEMM = 4, K_GSDOT = 5, K_NCLASS = 6 };
  struct Tick { cudaEvent_t a, b; int cls; double bytes, flops; };
  std::vector<Tick> pending_ticks;
  std::vector<cudaEvent_t> event_pool;
  int64_t launches[K_NCLASS] = {0, 0, 0, 0, 0, 0};
  double ms[K_NCLASS] = {0, 0, 0, 0, 0, 0};
  double bytes[K_NCLASS] = {0, 0, 0, 0, 0, 0};
  double flops[K_NCLASS] = {0, 0, 0, 0, 0, 0};
  int64_t kernel_launches = 0;
  // with opts.profile, every sample_every-th Arnoldi step and sweep runs eagerly and timed
  int sample_every() const { return opts.profile > 1 ? opts.profile : 8; }
  double setup_ms_total = 0;
  int last_columns = 0;
  int64_t sweep_calls = 0;
  bool sample_next_sweep = false;  // the next eager sweep times its GEMM steps one by one
  int ns_blocks = 0, ns_iterations = 0;  // strip inverses by Newton-Schulz, and its iterations
  int64_t iterations_total = 0;           // Arnoldi steps run (timed or replayed)
  int step_graphs_captured = 0;           // Arnoldi-step graphs captured
  bool step_graph_fallback = false;       // a step could not be captured
  Tick cur_tick[K_NCLASS];
  bool tick_open[K_NCLASS] = {false, false, false, false, false, false};

  // request loop (hh_submit / hh_poll)
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool worker_started = false, stopping = false;
  struct Request;
  std::deque<Request*> queue;
  std::mutex solve_mu;  // serialises solves on the engine (blocking calls vs request loop)
  SlotSolver* batch_solver = nullptr;  // reused by solve_batch_dev while the slot count repeats
  int batch_slots = 0;

  ~Engine();
  int init(double k, int n, int strips, uint32_t dirs, const hh_opts* o);
  int factor();

  // helpers
  int dmalloc(void** p, size_t bytes);
  void dfree(void* p);
  unsigned grid_for(size_t work, int threads = 256) const;
  cudaError_t launch_coop(const void* fn, int grid, int block, size_t smem, void** args, int grid_y = 1);
  int check_device_error(const char* where);
  void set_cuda_error(cudaError_t e, const char* where);
  void count_launch(int n = 1) { kernel_launches += n; }
  void tick_begin(int cls);
  void tick_end(int cls, double bytes, double flops);
  void collect_ticks();

  // operations (device pointers, column stride = m*m complex128)
  int apply_operator(int ncols, const double2* x, double2* y);
  int apply_preconditioner_dev(int dcode, int ncols, const double2* r, double2* z, bool single);
  int assemble_rhs(int nsrc, const double* src_host, double2* rhs);
  int solve_batch_dev(int nrhs, const double2* rhs, double2* x, double tol, hh_result* res);

  // sweep on packed columns (strip-interleaved layout, C columns): Rin -> V, W = corrections
  int run_sweep(const void* Rin, void* V, void* W, int C, bool single);
  // partial: split-K slices (or nullptr); allow_graph = false keeps the sweep eager (graph
  // instantiation may allocate, which the no-allocation entry point must not)
  // T0, T1: one-line interface arrays (nullptr: the handle's own)
  int run_sweep_untimed(const void* Rin, void* V, void* W, int C, bool single, void* partial,
                        size_t partial_bytes, bool allow_graph = true, void* T0 = nullptr, void* T1 = nullptr);
  int apply_preconditioner_noalloc(int dcode, int ncols, const double2* r, double2* z, bool single);
  // the launches of one sweep, untimed and without a graph of their own (for captures)
  int sweep_inline(const void* Rin, void* V, void* W, int C, bool single);
  // runs the tensor-core autotuner for C columns per strip if it has not run yet
  int ensure_tuned(int C);
  size_t sweep_elem() const { return precision == HH_PREC_FP32 ? 8 : 16; }
  size_t sweep_ws_bytes(int C) const;          // bytes of one packed sweep array
  double sweep_flops(int C, bool single) const;
  double sweep_bytes(int C, bool single) const;
  int factor_blocks() const { return bdir.total > 0 ? bdir.total : R + 3; }
  int inverse_columns();  // setup.cu: the blocks of bdir beyond G and K

  // sweep workspaces (grown on demand)
  void* w_rin = nullptr;
  void* w_v = nullptr;
  void* w_w = nullptr;
  void* w_partial = nullptr;   // split-K slices of the sweep GEMM steps
  void* w_t0 = nullptr;        // one-line arrays of the interface scans
  void* w_t1 = nullptr;
  size_t w_partial_bytes = 0;
  size_t sweep_partial_bytes(int C) const;
  size_t w_cap_cols = 0;
  int ensure_sweep_ws(int C);
};

// Result of one finished slot (see SlotSolver::iterate).
struct SlotDone {
  void* tag;
  int slot;
  hh_result res;
};

// Continuous-batching MPGMRES driver over S slots (krylov.cu).  Right-hand sides are
// admitted into free slots between iterations; every iteration advances all active slots
// by one block Arnoldi step with a single batched sweep over their columns; a slot that
// converges (or stops) is finalised and freed at once.  Not thread safe: one owner thread.
class SlotSolver {
 public:
  explicit SlotSolver(Engine& E);
  ~SlotSolver();
  SlotSolver(const SlotSolver&) = delete;
  SlotSolver& operator=(const SlotSolver&) = delete;
  int init(int slots);
  int free_slots() const;
  int busy() const;
  // b[q], x[q]: host or device pointers of one column each; returns the number admitted
  // (at most free_slots()), or -status.
  int admit(int count, const double2* const* b, double2* const* x, const double* tol, void* const* tags,
            int* slot_out);
  // One iteration of all active slots; appends the slots finished during it to out.
  int iterate(std::vector<SlotDone>& out);

 private:
  struct Impl;
  Impl* impl;
};

}  // namespace hh
