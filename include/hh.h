/*
 * hh.h -- C ABI of the GB300 multipreconditioned directional-sweep Helmholtz solver.
 *
 * Problem (Section 1, Eq. (1a)-(1b)):  Delta u + k^2 u = f in (0,1)^2,
 * du/dn - i k u = 0 on the boundary, discretised by P1 finite elements on the uniform
 * right-triangle mesh with n x n cells (every cell cut along its SW-NE diagonal).
 * Unknowns: the (n+1)^2 nodal values, node (i, j) at (i h, j h), h = 1/n, stored at
 * index g = j * (n + 1) + i.  The linear system is A u = b with
 * A = K - k^2 M - i k M_Gamma and b = -M f_I (load vector of the source).
 *
 * Preconditioners (Section 2, Eqs. (2)-(4)): for every selected direction d a double sweep
 * (forward then backward block Gauss-Seidel) over N = strips non-overlapping strips of
 * R = n / N node lines, the last strip visited owning one extra line.  The diagonal
 * blocks are impedance-modified strip matrices: the strip's block of A whose cell layer on
 * the already-swept side is replaced by the zeroth-order impedance condition of Eq. (4)
 * (an approximate Schur complement of the block LU factorisation that a sweep is).
 *
 * Krylov method (Section 3): selective flexible multipreconditioned GMRES, x0 = 0, the t
 * preconditioners applied concurrently every iteration; selection (Section 4): t = 2 ->
 * each preconditioner gets the other one's new basis vector, t > 2 -> all get the sum.
 *
 * Data conventions for every vector argument:
 *   complex128 interleaved (re, im) doubles, 2 * (n+1)^2 doubles per column, node order g;
 *   several columns are stored one after the other (column stride 2 * (n+1)^2 doubles).
 *   Pointers may be DEVICE pointers (cudaMalloc / torch CUDA tensors, on the handle's
 *   device) or HOST pointers (pageable or pinned); host buffers are copied in and out by
 *   the library inside the call.  The caller owns every buffer it passes.
 *
 * Errors: every entry point returns an hh_status; nothing is thrown across the ABI.  The
 * message of the most recent failure in the calling thread is in hh_last_error().
 */
#ifndef HH_H
#define HH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hh_handle hh_handle;
typedef uint64_t hh_ticket;

typedef enum {
  HH_OK = 0,
  HH_EINVAL = 1,       /* bad argument: n % strips != 0, R < 2, k <= 0, dirs == 0, NULL pointer, ... */
  HH_ENOMEM = 2,       /* device allocation failed or the factors do not fit in free device memory */
  HH_ENOCONV = 3,      /* maxit reached; x holds the best iterate */
  HH_EBREAKDOWN = 4,   /* every new direction deflated before convergence; x holds the iterate */
  HH_ENAN = 5,         /* NaN / Inf met in a norm */
  HH_ETIMEOUT = 6,     /* a bounded device-side wait ran out; the kernel returned early */
  HH_EPENDING = 7,     /* hh_poll: the ticket is not finished yet */
  HH_ECUDA = 8         /* a CUDA runtime call failed */
} hh_status;

/* direction bits (Section 4 vocabulary: the direction of the FORWARD pass) */
enum { HH_DIR_LR = 1, HH_DIR_RL = 2, HH_DIR_BT = 4, HH_DIR_TB = 8 };
enum { HH_PREC_FP64 = 0, HH_PREC_FP32 = 1, HH_PREC_BF16 = 2 };  /* precision of factors + sweeps */
enum { HH_SCHEME_AUTO = 0, HH_SCHEME_CROSS = 1, HH_SCHEME_SUM = 2 };
enum { HH_DISC_P1 = 0, HH_DISC_FD = 1 };  /* hh_opts.discretization */

typedef struct {
  int precision;          /* HH_PREC_FP64 (default) or HH_PREC_FP32: complex64 strip factors and
                             sweeps; HH_PREC_BF16: complex64 setup and sweep lines, but the factors
                             stored in bf16 and every sweep product ONE bf16 tensor-core MMA per K step
                             with FP32 accumulation (a cheaper, less accurate preconditioner: needs the
                             tensor cores and interface_form 1; odd column counts take the complex64
                             path); the global residual, Gram-Schmidt and Hessenberg stay FP64 */
  int scheme;             /* HH_SCHEME_AUTO: t=2 cross, t>2 sum */
  int single_sweep;       /* 1: forward sweeps only (LR, RL, BT, TB of Section 4) */
  int maxit;              /* iteration limit (default 200) */
  double deflate_eta;     /* deflation threshold r_jj <= eta * ||w_j|| (default 1e-10) */
  int bcr_depth;          /* the strip solves with a full right-hand side (w = D^{-1} r, every strip):
                             0 (default): block Thomas, 2R+1 dependent steps; d >= 1 (n / strips
                             divisible by 2^d): d levels of block cyclic (odd-even) reduction, then
                             block Thomas on the reduced system of R / 2^d lines, 2d + 2R/2^d + 1
                             dependent steps, every level one grouped step over its lines and all
                             strips; -1: the blocks of every usable depth are stored and the
                             fastest depth is picked by timing whole sweeps, per column count
                             (together with the twisted strip solves when they are stored, see
                             twisted); a fixed depth d >= 1 takes precedence over twisted */
  int64_t timeout_cycles; /* SM clock budget of every device-side wait (default 4e9) */
  void* stream;           /* cudaStream_t to run on, or NULL for the handle's own stream */
  int use_graph;          /* 1 (default): every Arnoldi step (table gather, pack, the sweep's
                             200-odd dependent launches, unpack, operator, Gram-Schmidt, block QR,
                             Givens update, next sources) is captured once per number of active
                             right-hand sides and replayed as a CUDA graph; sweeps run on their own
                             (hh_apply_preconditioner) are captured the same way */
  int profile;            /* 0: off; 1: time every kernel class with CUDA events (hh_get_stats), with
                             graphs on in every 8th Arnoldi step and sweep, which then run eagerly;
                             p > 1: the same in every p-th step and sweep */
  int gs_passes;          /* Gram-Schmidt passes against the basis and within the new block:
                             2 (default, CGS2) or 1 (the single pass whose inner products
                             Section 3 counts, (k - 1/2) t^2 + 3t/2 at iteration k) */
  int serve_slots;        /* slots of the hh_submit request loop: requests solved together,
                             each joining at an iteration boundary (default 8, 1..256) */
  int tensor_cores;       /* HH_PREC_FP32 only.  1 (default): the wide sweep steps run on the
                             tensor cores (tcgen05, TF32 operands split hi + lo, three products,
                             FP32 accumulation); 0: FP32 FMA on the CUDA cores */
  int autotune;           /* 1 (default): time the tensor-core step's tile shapes and K splits on
                             the first sweep of each column count and keep the fastest; 0: 64
                             complex columns per CTA, K split to fill the SMs (for runs under a
                             profiler, whose per-launch overhead would blur the timings);
                             -(1 + 7 s + v): candidate v (K split 0 = fill the SMs, 1, 2, 4 summed
                             by a reduction kernel; 2, 4, 8 summed in a thread-block cluster) of
                             shape s (0: 64 columns, 1: 32 columns, 2: 128 columns), for tests */
  int fuse_chains;        /* 1 (default): each interface chain of at most 8 columns (the N-2 and
                             N-1 dependent strip-to-strip steps of a double sweep) runs as one
                             cooperative launch that keeps its factor block in shared memory and
                             puts a grid barrier between the steps; 0: two launches per step */
  int overlap_steps;      /* 1 (default): each tensor-core sweep step is launched with programmatic
                             dependent launch, so that its prologue and first factor tiles overlap
                             the end of the preceding kernel (it waits for that kernel before it
                             reads the line data); 0: plain stream order */
  int interface_form;     /* how a sweep passes interface data from strip to strip (Section 2's
                             block forward / backward substitution, reorganised exactly):
                             1 (default): the interface recurrences of the forward and backward
                             passes as prefix-doubling scans (log2 N grouped steps over all
                             strips, with the powers G^(2^l), K^(2^l) of the strip transfer
                             blocks) and each pass's correction of the strips' interior lines as
                             ONE grouped step with stored block columns of the strip inverse;
                             0: chains of N-2 and N-1 dependent steps and block-Thomas corrections
                             (2R+1 and R-1 dependent steps) */
  int persistent;         /* HH_PREC_FP32 with the tensor cores, interface form 1, even column count:
                             1: the whole sweep (every phase of its program) runs as ONE cooperative
                             launch of one CTA per SM, grid barriers between the phases, factor and
                             line tiles streamed by TMA through a ring that runs on from one work item
                             to the next, two tensor-memory accumulators so that the epilogue of a
                             tile overlaps the MMAs of the next; 2: the same, reading the complex64
                             factor store once and splitting it into TF32 hi + lo in shared memory;
                             0 (default, faster at one right-hand side on this part): one launch per
                             phase, replayed as a CUDA graph */
  int gs_first_fp32;      /* HH_PREC_FP32 with two Gram-Schmidt passes: 1 (default): the inner
                             products of the FIRST pass against the basis in FP32 (their
                             coefficients are applied in FP64 and the FP64 second pass corrects
                             them, so H, the orthogonality of V and A Z = V H stay FP64-accurate);
                             0: both passes in FP64 */
  int discretization;     /* HH_DISC_P1 (default): P1 finite elements on the right-triangle mesh and
                             non-overlapping strips; HH_DISC_FD: the paper's own setting (Section 4),
                             five-point finite differences with ghost-node Robin rows and strips
                             overlapping by 2h that exchange Robin data, every node taking the most
                             recent subdomain solve; FP64 only (HH_PREC_FP64), sweeps on the CUDA cores */
  int group_wide_tiles;   /* complex64 tensor-core sweeps: 1 (default): a grouped step whose tasks are
                             wider than 64 columns and at most 128 and whose tiles fill the SMs
                             without a K split (the one-shot corrections of interface form 1 at
                             one right-hand side) runs with 128-column tiles, reading each factor
                             tile once, and a step whose tasks are all within 32 columns with
                             32-column tiles; 0: the autotuned line-step shape */
  int gs_tensor;          /* 1 (default): the inner products and updates of Gram-Schmidt against the
                             basis run on the tensor cores as exact integer products of 7-bit slices
                             of the FP64 data (FP64-accurate; about 64 more bytes of device memory
                             per node for every basis vector); 0: on the FP64 pipe */
  int twisted;            /* the strip solves with a full right-hand side by a twisted block
                             factorisation (complex64 tensor-core sweeps, interface_form 1,
                             strips >= 2, n / strips >= 4, bcr_depth <= 0; other sweeps, bf16
                             ones included, keep block Thomas or the fixed depth): the
                             first R = n / strips lines of every strip are eliminated from both
                             ends at once, meeting at line R/2, so that each dependent step carries
                             a top and a bottom task and the chain is R + 1 steps instead of
                             2R + 1, with the same factor bytes; the last strip's extra line R
                             follows by its Schur complement after the interface corrections.
                             It needs 2 + R/2 more m x m blocks, whose setup takes longer (their
                             Newton-Schulz iterations start farther from the inverse: 58 ms more
                             at k = 400, n = 1024), and saves 13 % of every sweep there.
                             1 (default): used; -1: stored and timed against block Thomas (and
                             the stored cyclic-reduction depths) per column count; 0: not stored
                             (streams of problems that are each solved once) */
} hh_opts;

typedef struct {
  int iterations;             /* MPGMRES iterations (each adds up to t search directions) */
  double rel_res_implicit;    /* |g_last| / ||b|| from the Hessenberg least-squares problem */
  double rel_res_explicit;    /* ||b - A x|| / ||b|| recomputed in FP64 on the device */
  double t_setup_ms, t_solve_ms;
  hh_status status;
} hh_result;

typedef struct {
  /* per kernel class: launches, summed device time (ms, only with opts.profile) and the
     algorithmic bytes those launches must move (the roofline model of each kernel) */
  int64_t sweep_launches;  double sweep_ms;  double sweep_bytes;
  int64_t spmv_launches;   double spmv_ms;   double spmv_bytes;
  int64_t gs_launches;     double gs_ms;     double gs_bytes;
  int64_t setup_launches;  double setup_ms;  double setup_flops;
  int64_t kernel_launches; /* every kernel this handle launched */
  int64_t factor_bytes;    /* device bytes of the stored strip factors */
  int factor_blocks;       /* distinct m x m blocks stored (R + 1) */
  int m, ldf, columns;     /* nodes per line, padded leading dimension, sweep columns of last solve */
  int64_t sweep_steps;     /* dependent block steps of one sweep launch */
  /* the wide GEMM steps of the sweeps, timed one by one in every sampled sweep (see
     opts.profile): sampled launches, their device time (ms) and their complex
     multiply-add flops (8 m^2 per column) */
  int64_t gemm_launches;   double gemm_ms;   double gemm_flops;
  int tensor_cores;        /* 1 when the wide sweep steps run on the tensor cores */
  /* the Gram-Schmidt inner-product kernel (every launch, within the gs class): launches,
     device time (ms, with opts.profile) and FP64 flops (8 per basis element and new column) */
  int64_t gsdot_launches;  double gsdot_ms;  double gsdot_flops;
  double gs_flops;         /* FP64 flops of the whole gs class (both passes, dot + update) */
  int64_t wide_steps;      /* wide GEMM steps in one sweep of the last column count */
  int ns_blocks;           /* strip inverses computed by Newton-Schulz from the previous one */
  int ns_iterations;       /* their iterations (two GEMMs each) */
  int tc_bnc, tc_nsplit;   /* autotuned tensor-core step for the last column count: complex
                              columns per CTA (64, 32 or 128) and K split (0 = fill the SMs) */
  int tc_cluster;          /* 1 when its K slices are summed in a thread-block cluster */
  double tc_us;            /* its time per step when tuned (us; a run of consecutive steps) */
  int64_t iterations_total; /* Arnoldi steps run, timed or replayed from their graph (with
                               opts.profile the classes above time the sampled steps) */
  int step_graphs;          /* Arnoldi-step graphs captured by the handle's solvers */
  int step_graph_fallback;  /* 1 if a step could not be captured and ran eagerly */
  int bcr_depth;            /* cyclic-reduction depth of the strip solves for the last column
                               count (fixed by opts.bcr_depth or autotuned) */
  double gsdot_bytes;       /* algorithmic bytes of the timed inner-product launches (the
                               tensor-core form: the basis slice images and the new columns,
                               read once) */
  int twisted;              /* 1 when the strip solves of the last column count use the twisted
                               factorisation (opts.twisted) */
} hh_stats;

/* Fill *o with the defaults listed above. */
void hh_default_opts(hh_opts* o);

/*
 * Assemble nothing on the host: validate, allocate the factor store and run the strip
 * setup on the device (Section 2: block LU of each strip; the Schur complements
 * S_0 = D_bot, S_j = D_int - L S_{j-1}^{-1} U and their dense inverses).  Strips of equal
 * size have equal matrices, so the R + 1 distinct m x m inverses are computed and stored
 * once (m = n + 1).  dirs is a bitmask of HH_DIR_*; t = popcount(dirs).
 * Errors: HH_EINVAL (n % strips, n / strips < 2, k <= 0, dirs == 0, n > 4096, out == NULL),
 * HH_ENOMEM, HH_ECUDA, HH_ETIMEOUT.  On success *out owns device memory until hh_destroy.
 */
hh_status hh_setup(double k, int n, int strips, uint32_t dirs, const hh_opts* opts, hh_handle** out);

/* Solve A x = rhs to relative residual tol (Section 3, 4).  Blocking.  rhs, x: one column.
 * x is written for HH_OK, HH_ENOCONV and HH_EBREAKDOWN; res may be NULL. */
hh_status hh_solve(hh_handle* h, const double* rhs, double* x, double tol, hh_result* res);

/* nrhs independent solves sharing every sweep launch (columns batched): rhs and x hold
 * nrhs columns; res (may be NULL) receives nrhs results.  Returns the worst status. */
hh_status hh_solve_batch(hh_handle* h, int nrhs, const double* rhs, double* x, double tol,
                         hh_result* res);

/* Asynchronous solve: queued on the handle's request loop (continuous batching: requests
 * that share a handle join the next iteration's sweep launch as columns free up).
 * rhs and x must stay valid until hh_poll returns something other than HH_EPENDING. */
hh_status hh_submit(hh_handle* h, const double* rhs, double* x, double tol, hh_ticket* ticket);

/* Never blocks.  HH_EPENDING while the ticket runs; otherwise the request's final status
 * (and *res if res != NULL); a finished ticket can be polled once more, then it is freed. */
hh_status hh_poll(hh_ticket ticket, hh_result* res);

/* Load vector b = -M f_I of a sum of Gaussians (the benchmark source family of Section 4):
 * src holds nsrc rows (x0, y0, sigma, amp_re, amp_im), HOST memory; rhs one column. */
hh_status hh_assemble_rhs(hh_handle* h, int nsrc, const double* src, double* rhs);

/* y = A x for ncols columns (FP64, matrix-free seven-point stencil of the P1 matrix). */
hh_status hh_apply_operator(hh_handle* h, int ncols, const double* x, double* y);

/* z = M_d^{-1} r for ncols columns and ONE direction bit (the handle's precision; a double
 * sweep unless opts.single_sweep).  dir need not be in the handle's dirs. */
hh_status hh_apply_preconditioner(hh_handle* h, uint32_t dir, int ncols, const double* r, double* z);

/* One pass of the block classical Gram-Schmidt of Section 3 against p basis columns, with the
 * solver's kernels (hh_opts.gs_tensor of the handle selects the tensor-core slices or the
 * FP64 pipe): H = V^H W, then W <- W - V H.
 *   V  p complex128 columns of (n+1)^2 entries (column stride 2 (n+1)^2 doubles), host or device;
 *   W  t complex128 columns (1 <= t <= 4), host or device, overwritten with W - V H;
 *   H  HOST memory, p x t complex128, entry (a, b) at 2 (a t + b): <v_a, w_b> = sum conj(v_a) w_b.
 * Allocates its working buffers (the slice images: 64 bytes per node per basis column) for the
 * call.  HH_EINVAL for p < 1, t outside 1..4 or a NULL pointer. */
hh_status hh_gram_schmidt_pass(hh_handle* h, int p, const double* V, int t, double* W, double* H);

/*
 * z = M_d^{-1} r like hh_apply_preconditioner, for callers that cannot allocate device
 * memory during the call (a device-memory budget fixed at start-up, a host framework whose
 * caching allocator owns the device, or a latency-critical path that must avoid cudaMalloc
 * and cudaFree and the device synchronisation they can cause).  The paper has no
 * counterpart: this is a deployment variant of the sweep entry point.
 *   - allocates nothing: no cudaMalloc / cudaFree and no allocating library routine; its
 *     scratch is a fixed 32 MiB device array inside the library, present on every GPU the
 *     library is loaded on until the process exits;
 *   - r and z must be DEVICE pointers (ncols complex128 columns); host pointers -> HH_EINVAL;
 *   - a grid / column count whose packed sweep arrays exceed the 32 MiB -> HH_EINVAL
 *     (roughly: complex64 factors up to n = 512 with 4 columns, n = 1024 not at all);
 *   - hh_setup resolves the array's device address once per device (which also loads the
 *     module holding it, so that the array is reserved on the device from then on); this
 *     entry point itself only reads that address;
 *   - every call shares the one array and leaves its contents behind; nothing in it needs to
 *     start at zero; calls whose GPU work overlaps (other handles, other streams, other
 *     threads) race on it and must be serialised by the caller.
 */
hh_status hh_apply_preconditioner_noalloc(hh_handle* h, uint32_t dir, int ncols, const double* r, double* z);

/* Copy block j of the factor store as complex128 row-major m x m into out: j = 0..R the
   block-Thomas inverses S_j^{-1} (Section 2's strip solves); j = R+1 .. factor_blocks-1 (see
   hh_stats) the blocks derived from them in the order of the store; with the twisted strip
   solves (hh_opts.twisted) the last R/2 + 1 blocks are G_{R/2+1} .. G_{R-1}, M and Z_0. */
hh_status hh_get_factor(hh_handle* h, int j, double* out);

hh_status hh_get_stats(hh_handle* h, hh_stats* st);
void hh_reset_stats(hh_handle* h);

/* Release every device resource of the handle (pending tickets are cancelled). */
void hh_destroy(hh_handle* h);

/* Message of the last failure in this thread ("" if none).  Valid until the next call. */
const char* hh_last_error(void);

/* ---------------------------------------------------------------------------------------
 * Serving: requests for many problems (k, n) behind one submit / poll interface.
 *
 * The server keeps one handle per (k, n, strips, dirs) resident on the device (strip
 * factors, sweep workspaces, Krylov state) and reuses it for later requests of the same
 * problem.  A request for an uncached problem is admitted by device memory: the new
 * handle's bytes are estimated and, if the budget is exceeded, idle handles are evicted least
 * recently used first; if that is not enough the request waits until running requests
 * finish.  Each handle has its own stream and request loop (continuous batching, hh_submit),
 * so solves of different problems and the setup of a new one overlap on the device.
 * ------------------------------------------------------------------------------------- */
typedef struct hh_server hh_server;

typedef struct {
  int64_t handles;          /* problems resident */
  int64_t bytes_reserved;   /* estimated device bytes of the resident handles */
  int64_t budget;           /* device-memory budget */
  int64_t setups;           /* handles built */
  int64_t cache_hits;       /* requests served by a resident handle */
  int64_t evictions;        /* handles destroyed to make room */
  int64_t completed;        /* requests finished */
  int64_t queued, running;  /* requests waiting for admission / being solved */
  double setup_ms;          /* summed host time of the setups */
} hh_server_stats;

/* opts: the options of every handle the server builds (NULL = defaults; the stream field
 * is ignored: every handle gets its own).  A stream whose problems are mostly distinct, each
 * solved a few times, is better served with twisted = 0: the twisted strip solves' extra
 * setup (58 ms at k = 400, n = 1024) outweighs what they save per solve (about 5 ms there).
 * mem_budget: device bytes the resident handles may hold (0 = 85 % of the free device memory
 * at creation).  Errors: HH_EINVAL, HH_ECUDA. */
hh_status hh_server_create(const hh_opts* opts, size_t mem_budget, hh_server** out);

/* Queue one solve of the problem (k, n, strips, dirs) with the load vector of nsrc Gaussian
 * sources (rows x0, y0, sigma, re, im; copied) to relative residual tol.  x: host or device
 * pointer of 2 (n+1)^2 doubles (complex128, node order), written when the request finishes;
 * it must stay valid until hh_server_poll returns something other than HH_EPENDING.
 * Errors: HH_EINVAL (bad problem or arguments). */
hh_status hh_server_submit(hh_server* s, double k, int n, int strips, uint32_t dirs, int nsrc, const double* src,
                           double* x, double tol, hh_ticket* ticket);

/* HH_EPENDING while the request is queued or running; otherwise its final status, with
 * res->t_solve_ms = time from submission to completion (queueing, setup and solve) and
 * res->t_setup_ms the problem's setup time. */
hh_status hh_server_poll(hh_server* s, hh_ticket ticket, hh_result* res);

hh_status hh_server_get_stats(hh_server* s, hh_server_stats* st);

/* Fails the queued requests (HH_EINVAL), waits for the running ones, frees everything. */
void hh_server_destroy(hh_server* s);

#ifdef __cplusplus
}
#endif
#endif /* HH_H */
