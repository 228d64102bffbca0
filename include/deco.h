/*
 * deco.h -- C ABI of the GB300 (sm_103a) hot path of the DECO MaxCut solver
 * ("A Scalable Lift-and-Project Differentiable Approach For the Maximum Cut
 * Problem", arXiv 2509.18612).
 *
 * The library computes batched projected gradient ascent (PGA) on the relaxed
 * cut objective over an n x C block of starting points, alternating unlifted
 * (Eq. QUCO, Alg. 1) and lifted (Eq. LUCO, Alg. 2) phases as in Alg. 3, then
 * rounds every column (Eq. 5 / Eq. 11), evaluates integer cut values (Eq. 1)
 * and takes the argmax over starting points.
 *
 * Conventions shared by every entry point
 *  - All functions return an int status: DECO_OK (0) or a negative
 *    deco_status code.  On error the outputs are left untouched and
 *    deco_last_error() returns a message (thread-local).  No C++ exception
 *    crosses this boundary.
 *  - Pointers documented as "device" must be CUDA device (or managed)
 *    memory of the current device; "host" pointers are plain host memory.
 *    The caller owns every buffer it passes in; the library never frees them.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    stream-ordered; functions that return host results synchronise the
 *    stream before returning.
 *  - Iterates are stored in *centred* coordinates y in [-1,1], row-major
 *    n x ld (column c of row v at y[v*ld + c]); ld >= C, ld % 8 == 0.
 *    For the multilinear objective the paper-facing variable is x = (1+y)/2.
 *    Columns of a lifted block are grouped per starting point: column
 *    b*l + i holds component i of starting point b.
 *  - Element types: DECO_PREC_FP32 -> float, DECO_PREC_BF16 -> 16-bit
 *    bfloat16 (round to nearest even on store; all arithmetic in FP32).
 */
#ifndef DECO_H_
#define DECO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DECO_ABI_VERSION 2

typedef enum deco_status {
  DECO_OK = 0,
  DECO_ERR_ARG = -1,         /* invalid argument (NULL pointer, bad size, bad enum) */
  DECO_ERR_GRAPH = -2,       /* malformed CSR (see deco_create_graph) */
  DECO_ERR_OOM = -3,         /* device allocation failed */
  DECO_ERR_CUDA = -4,        /* a CUDA runtime call failed */
  DECO_ERR_NONFINITE = -5,   /* a non-finite value appeared in the iterate */
  DECO_ERR_TIMEOUT = -6,     /* a bounded device wait gave up */
  DECO_ERR_UNSUPPORTED = -7  /* valid request this build does not implement */
} deco_status;

/* Objectives (both in centred coordinates y in [-1,1]^n).
 * DECO_OBJ_MULTILINEAR01: F(x) = sum_{(i,j) in E} w_ij (x_i + x_j - 2 x_i x_j)
 *   on x in [0,1]^n, gradient d - 2 A x; the step
 *   x <- Proj[0,1](x + alpha (d - 2 A x)) equals y <- Proj[-1,1](y - 2 alpha A y).
 * DECO_OBJ_LAPLACIAN: f(x) = x^T L x on [-1,1]^n (Eq. QUCO), g = L x (Eq. 6),
 *   step x <- Proj[-1,1](x + alpha L x) (Eq. 7; Eq. 10 per column when lifted). */
#define DECO_OBJ_MULTILINEAR01 0
#define DECO_OBJ_LAPLACIAN 1

#define DECO_PREC_FP32 0
#define DECO_PREC_BF16 1

/* Initialisation of the first phase (Sec. 4.1, 4.2 and 5 of the paper).
 *  UNIFORM          y = h * (2u - 1), u ~ U(0,1), h = uniform_half_width
 *  IDI              Gaussian around h_IDI (Sec. 4.1.2)
 *  DUI              Gaussian around h_DUI (Eq. 12)
 *  IDI_HALF_UNIFORM starting points [0, B/2) as IDI, [B/2, B) as
 *                   scale * (2u - 1)
 *  EXPLICIT         caller-given x0 in the objective's own domain
 *                   ([0,1] multilinear, [-1,1] Laplacian)
 *  MEAN             Gaussian around a caller-given mean h (device, n floats)
 * "Gaussian around h": y = Proj[-1,1](scale * (h_v + sqrt(eta) * N(0,1))).
 * Every later phase is Gaussian around 2 z* - 1, z* the previous phase's best
 * binary vector (Sec. 4.2; Alg. 3). */
#define DECO_INIT_UNIFORM 0
#define DECO_INIT_IDI 1
#define DECO_INIT_DUI 2
#define DECO_INIT_IDI_HALF_UNIFORM 3
#define DECO_INIT_EXPLICIT 4
#define DECO_INIT_MEAN 5

/* Kernel used for the steps of a phase.
 *  AUTO    the persistent on-chip kernel when a 128-byte column slab of the
 *          graph (plus its share of the CSR) fits in shared memory, else one
 *          launch of the global-memory kernel per step
 *  GLOBAL  always the per-step global-memory kernel
 *  ONCHIP  always the persistent on-chip kernel (DECO_ERR_UNSUPPORTED if it
 *          does not fit)
 *  DENSE   (BF16 blocks) the tensor-core kernel for dense graphs: A Y as a
 *          dense BF16 x BF16 -> FP32 product on the 5th-generation tensor
 *          cores (tcgen05, accumulator in tensor memory) with the update
 *          fused into the epilogue; needs |w| <= 256, n <= 32768 and C <= 1024.
 *          The dense copy of A (round_up(n,128)^2 BF16 values) is built on
 *          first use and kept with the graph.  FP32 blocks (e.g. the FP32
 *          polish of deco_solve) are planned as with AUTO.  Never chosen by
 *          AUTO's cost model, only by the autotuner or explicitly.
 * GLOBAL and ONCHIP perform the same FP32 operations in the same order, so
 * their iterates are bit-identical.  DENSE sums each row of A Y in the
 * tensor cores' order (and, with k > 1, k partial sums in rank order): its
 * iterates agree with the others to FP32 summation error, and are
 * reproducible from run to run. */
#define DECO_KERNEL_AUTO 0
#define DECO_KERNEL_GLOBAL 1
#define DECO_KERNEL_ONCHIP 2
#define DECO_KERNEL_DENSE 3
/* With DECO_KERNEL_ONCHIP, DECO_KERNEL_CLUSTER(k) (k = 1, 2, 4 or 8) fixes the
 * cluster size instead of the built-in cost model's choice.  With
 * DECO_KERNEL_DENSE it fixes the split of the contraction over k CTAs of a
 * cluster (k partial products reduced through distributed shared memory). */
#define DECO_KERNEL_CLUSTER(k) ((k) << 8)
/* With DECO_KERNEL_DENSE, one launch per step instead of the persistent phase
 * kernel (one cooperative launch per phase, a grid barrier between steps, used
 * when all its CTAs can be resident at once). */
#define DECO_KERNEL_DENSE_PER_STEP (1 << 12)
/* With DECO_KERNEL_ONCHIP, fixes the CTA size of the on-chip kernel. */
#define DECO_KERNEL_THREADS_512 (1 << 12)
#define DECO_KERNEL_THREADS_1024 (2 << 12)
/* With DECO_KERNEL_ONCHIP and a cluster of more than one CTA, fixes how the
 * CTAs exchange their new rows after every step: through distributed shared
 * memory stores, or through L2 (global stores + one bulk copy per CTA). */
#define DECO_KERNEL_EXCHANGE_DSMEM (1 << 14)
#define DECO_KERNEL_EXCHANGE_L2 (2 << 14)
/* With DECO_KERNEL_GLOBAL, runs the block as 2^s column slabs (s = 1..6; a 3-bit field), one
 * after another: the block is copied into dense n x w slabs (w = C / 2^s
 * rounded up to 8) and every step of a slab runs before the next slab, so a
 * narrow slab of a graph too large for shared memory stays in L2.  Needs
 * ld >= round_up(C, 8 * 2^s). */
#define DECO_KERNEL_COLUMN_SLABS(s) ((s) << 16)
/* With DECO_KERNEL_ONCHIP, the lean form: no staging area in shared memory
 * and the momentum kept in global memory, the new rows exchanged through L2
 * (also by a single CTA), so that a cluster half as large fits.  Same
 * iterates as the other forms. */
#define DECO_KERNEL_LEAN (1 << 20)
/* With DECO_KERNEL_ONCHIP, the row-pair form: each half of a warp works on its
 * own row (every lane on 8 bytes of the 128-byte replica row), so a warp
 * advances two rows at a time and one shared load serves an entry of each.
 * Same iterates as the other forms.  DECO_KERNEL_AUTO without a recorded
 * tuning, and the batched on-chip launch of deco_solve_batch, use this form. */
#define DECO_KERNEL_ROW_PAIRS (1 << 21)
/* With DECO_KERNEL_GLOBAL (optionally with column slabs), the pipelined form
 * of the per-step kernel: rows sorted by degree in slices of 32 / G rows (G
 * lanes per row, 16 bytes of the row per lane); slice s belongs to warp
 * s mod #warps, whose items (a slice, or a part of `entries` entries of a
 * slice with longer rows) form one contiguous stream of fixed-size records
 * (rows, counts, padded column indices), built on first use for the graph and
 * launch shape and kept with the graph.  A warp copies each record into shared
 * memory (cp.async) 2S - 1 items ahead and the neighbour rows of each item
 * S - 1 items ahead, and sums an item's rows in CSR order from shared memory.
 * Same iterates as the other forms.  Its shape:
 *   DECO_KERNEL_PIPE_ENTRIES(e)  entries of a row per item: e = 0: 16,
 *                                1: 8, 2: 24, 3: 12 (longer rows go in parts)
 *   DECO_KERNEL_PIPE_STAGES(s)   shared-memory stages per warp: s = 0: 3,
 *                                1: 2, 2: 4
 *   DECO_KERNEL_PIPE_WARPS(w)    warps per block: w = 0: as many as fit
 *                                (at most 8), 1..7: w
 * The shapes with 8 or 12 entries in 2 stages run a form of the kernel
 * compiled for that shape (loops fully unrolled); the others read the shape
 * at run time. */
#define DECO_KERNEL_PIPELINED (1 << 22)
#define DECO_KERNEL_PIPE_ENTRIES(e) ((e) << 23)
#define DECO_KERNEL_PIPE_STAGES(s) ((s) << 25)
#define DECO_KERNEL_PIPE_WARPS(w) ((w) << 27)
/* With DECO_KERNEL_PIPELINED and BF16 blocks of unit-weight graphs: the sums
 * use Blackwell's mixed-precision add (BF16 operand widened exactly, one FP32
 * rounding), the same operation as widening first and adding. */
#define DECO_KERNEL_PIPE_MIXED_ADD (1 << 30)
/* With DECO_KERNEL_PIPELINED: the records and the new rows are read and
 * written with the L2 evict-first priority, so that L2 keeps the block (or
 * column slab) being gathered.  Same iterates. */
#define DECO_KERNEL_PIPE_L2_HINTS (1 << 19)
/* With DECO_KERNEL_PIPELINED: the wide form, each lane carrying two 16-byte
 * vectors of its row, so an item holds twice the rows for the same columns
 * (half the items per step).  Runs the shapes with 8 or 12 entries per item
 * in 2 stages (DECO_ERR_UNSUPPORTED otherwise).  Same iterates. */
#define DECO_KERNEL_PIPE_WIDE (1 << 2)

/* deco_create_graph flags */
#define DECO_GRAPH_SKIP_SYMMETRY_CHECK 0x1u  /* caller guarantees symmetry */

typedef struct deco_graph deco_graph;

/* Create a graph from a symmetric CSR (both orientations stored).
 * Def. 1 / Eq. 1 of the paper (undirected graph, cut counts each crossing
 * edge once); Sec. 2 notation for A, D, L.
 *  n        >= 1 nodes; nnz >= 0 stored entries (= 2 m), nnz < 2^31.
 *  row_ptr  host, n+1 int32, row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz.
 *  col_idx  host, nnz int32 in [0,n), strictly increasing within each row,
 *           no self loops; (u,v) present iff (v,u) present.
 *  weights  host, nnz floats or NULL (unit weights).  Every weight must be a
 *           nonzero integer with |w| <= 2^20 and w(u,v) = w(v,u) (cut values
 *           are computed exactly in integers).
 *  flags    DECO_GRAPH_* bits.
 *  out      receives the handle; the library copies everything it needs to
 *           the current device (the caller's arrays may be freed afterwards).
 * Errors: DECO_ERR_ARG (NULL/size), DECO_ERR_GRAPH (validation; message says
 * which rule and where), DECO_ERR_UNSUPPORTED (non-integral weights),
 * DECO_ERR_OOM / DECO_ERR_CUDA.  Validation happens before any CUDA call. */
int deco_create_graph(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                      const float* weights, uint32_t flags, deco_graph** out);

/* Release a graph (NULL is a no-op). */
void deco_destroy_graph(deco_graph* g);

/* Graph facts: n, nnz, and whether weights are present (1) or unit (0). */
int deco_graph_info(const deco_graph* g, int32_t* n, int64_t* nnz, int32_t* weighted);

/* Integer cut value of one binary vector (Def. 1, Eq. 1):
 *   Cut = sum over unordered edges {u,v} with z_u != z_v of w_uv.
 *  z        host, n bytes, each 0 or 1 (any nonzero byte counts as 1).
 *  cut_out  host, receives the exact value.
 * Synchronous.  Errors: DECO_ERR_ARG, DECO_ERR_OOM, DECO_ERR_CUDA. */
int deco_eval_cut(const deco_graph* g, const uint8_t* z, int64_t* cut_out);

/* Batched integer cut values (Eq. 1) of B binary columns.
 *  z     device, n x B bytes row-major (z[v*B + b]), 0/1.
 *  cuts  device, B int64 (overwritten).  Stream-ordered, asynchronous. */
int deco_eval_cuts(const deco_graph* g, int32_t B, const uint8_t* z, int64_t* cuts, void* stream);

/* Arguments of one fused PGA step.  Reading of the momentum form (the paper
 * only says momentum PGA is used, Sec. 4.2): heavy ball,
 *   V <- mu V + grad;  y <- Proj(y + alpha_eff V),
 * with grad = d (.) y - A y (Laplacian, alpha_eff = alpha) or grad = -A y
 * (multilinear, alpha_eff = 2 alpha). */
typedef struct deco_step_args {
  int32_t objective;          /* DECO_OBJ_* */
  int32_t precision;          /* DECO_PREC_* of y_in / y_out */
  float alpha;                /* step size when alpha_cols == NULL */
  float momentum;             /* mu; 0 = plain PGA (v ignored, may be NULL) */
  const float* alpha_cols;    /* device, C floats or NULL: per-column step size */
  const int32_t* steps_cols;  /* device, C int32 or NULL: column c is active
                                 only while t < steps_cols[c] (population search) */
  int32_t t;                  /* step index used with steps_cols */
  int32_t reserved;
} deco_step_args;

/* One projected gradient ascent step on every column (Eq. 7; Eq. 10 when the
 * block is lifted -- each column updates independently, remark after Eq. 11).
 *  C       columns, 1 <= C <= ld; ld % 8 == 0.
 *  y_in    device, n x ld, precision a->precision; not modified.
 *  y_out   device, n x ld, must not alias y_in; columns >= C untouched.
 *  v       device, n x ld float (momentum buffer, FP32 always), updated in
 *          place; may be NULL when a->momentum == 0.
 *  nonfinite_flag  device int32 or NULL: set to 1 if any new value is not
 *          finite (the value written is then clamped; the caller decides).
 * Stream-ordered, asynchronous.  Errors: DECO_ERR_ARG. */
int deco_step(const deco_graph* g, int32_t C, int32_t ld, const void* y_in, void* y_out,
              float* v, const deco_step_args* a, int32_t* nonfinite_flag, void* stream);

/* `steps` projected gradient ascent steps in place (the step loop of Alg. 1 /
 * Alg. 2): y holds the starting block and receives the result.
 *  C, ld   as in deco_step; the on-chip kernel needs ld % 32 == 0 (FP32) or
 *          ld % 64 == 0 (BF16) and treats columns in [C, ld) as inactive.
 *  v       device n x ld float momentum, read at the start and written at the
 *          end (NULL when a->momentum == 0).
 *  a       step arguments; a->t is ignored (step t runs t = 0 .. steps-1).
 *  kernel  DECO_KERNEL_* (with the optional modifiers above).
 *  nonfinite_flag  device int32 or NULL: bit 0 set if a new value is not
 *          finite; bit 1 set if a bounded wait of the on-chip or dense kernel
 *          gave up (the block is then unreliable).
 * Stream-ordered and asynchronous; scratch memory (exchange buffers, the
 * second block of the global kernel) is allocated and released in stream
 * order.  The first use of a graph with a given cluster size builds its
 * on-chip CSR image on the host (kept with the graph).
 * Errors: DECO_ERR_ARG, DECO_ERR_UNSUPPORTED (ONCHIP does not fit, DENSE
 * outside its limits), CUDA. */
int deco_run_phase(const deco_graph* g, int32_t C, int32_t ld, void* y, float* v, int32_t steps,
                   const deco_step_args* a, int32_t kernel, int32_t* nonfinite_flag, void* stream);

/* Autotuner: times every feasible launch shape of a phase on this graph --
 * the per-step global kernel, the on-chip kernel for each cluster size
 * (1, 2, 4, 8), CTA size (512, 1024) and exchange mode (DSMEM, L2), and, for
 * BF16 blocks of graphs with nnz >= n^2 / 64 inside the DENSE limits, the
 * tensor-core kernel for each contraction split (1, 2, 4, 8) -- over
 * `probe_steps` steps of a C-column block with the given precision,
 * objective and momentum, and records the fastest with the graph.  Later
 * deco_solve / deco_run_phase calls with DECO_KERNEL_AUTO on a block of the
 * same C and precision use the recorded shape instead of the cost model.
 *  best_kernel        host, receives the winning DECO_KERNEL_* selector.
 *  best_us_per_step   host, receives its time per step (microseconds).
 * Allocates and frees its own probe blocks; synchronous.
 * Errors: DECO_ERR_ARG, DECO_ERR_OOM, DECO_ERR_CUDA. */
int deco_autotune(const deco_graph* g, int32_t C, int32_t precision, int32_t objective, float momentum,
                  int32_t probe_steps, int32_t* best_kernel, float* best_us_per_step, void* stream);

/* Record a launch shape for (C, precision) on this graph without timing it
 * (e.g. one loaded from a saved tuning table); `kernel` must be a valid
 * DECO_KERNEL_* selector.  Errors: DECO_ERR_ARG. */
int deco_set_tuning(const deco_graph* g, int32_t C, int32_t precision, int32_t kernel);

/* deco_run_phase for callers that cannot let the library allocate device
 * memory: a host program whose own pool already holds (nearly) all of the
 * device, or a latency-bound loop where a cudaMalloc/cudaFree, which may
 * synchronise the device, is not acceptable.  The paper has no counterpart;
 * this is a deployment variant of the per-step phase runner above.
 *  Same arguments as deco_run_phase, always on the per-step global-memory
 *  kernel.  Results equal deco_run_phase with DECO_KERNEL_GLOBAL.
 *  Scratch: the second block of the step ping-pong lives in one fixed
 *  16 MiB device array inside the library (every GPU that loads the library
 *  keeps it until the process exits); n * ld * element size must not exceed
 *  16 MiB, otherwise DECO_ERR_UNSUPPORTED with a message, and nothing runs.
 *  No cudaMalloc, cudaFree or other allocating call is made.
 *  The first call on a device looks up the array's device address
 *  (cudaGetSymbolAddress); make that first call before any stream capture.
 *  The address is kept with the unique id of the CUDA context it belongs to;
 *  the first call after the context was torn down and re-created (e.g. by
 *  cudaDeviceReset) looks it up again, so it too must come before a capture.
 *  All calls share the one array: calls whose work overlaps on the GPU (other
 *  streams, other host threads) race on it and must be serialised by the
 *  caller.  Nothing in the array needs to start at zero.
 * Errors: DECO_ERR_ARG, DECO_ERR_UNSUPPORTED, DECO_ERR_CUDA. */
int deco_run_phase_noalloc(const deco_graph* g, int32_t C, int32_t ld, void* y, float* v, int32_t steps,
                           const deco_step_args* a, int32_t* nonfinite_flag, void* stream);

/* Rounding + cut + argmax of a block (the rounding and selection steps of
 * Alg. 1 / Alg. 2).
 *  B, lift  starting points and lift l (C = B*l columns in y, ld >= C).
 *  y        device, n x ld, precision `precision`.
 *  zbits    device, n x ceil(B/32) uint32 (bit b%32 of word b/32 = z_{v,b}):
 *           lift 1: z = 1{y > 0} (Eq. 5); lift l: z = 1{sum_i y_{v,bl+i} >= 0}
 *           (Eq. 11, summed in FP32 in order i = 0..l-1).
 *  cuts     device, B int64: cut of every starting point (Eq. 1).
 *  best     device, 1 int32: lowest index among the maximal cuts, or NULL.
 * Stream-ordered, asynchronous. */
int deco_round_cut(const deco_graph* g, int32_t B, int32_t lift, int32_t ld, int32_t precision,
                   const void* y, uint32_t* zbits, int64_t* cuts, int32_t* best, void* stream);

/* Starting block of phase `phase` (Sec. 4.1, 4.2, 5).
 *  init     DECO_INIT_*; for phases > 0 use DECO_INIT_MEAN with the previous
 *           best vector mapped to 2z-1.
 *  mean     device, n floats (DECO_INIT_MEAN) or NULL.
 *  x0       device, n x ld floats (DECO_INIT_EXPLICIT) or NULL.
 *  y        device, n x ld output block in `precision`.
 * Random draws: Philox4x32-10 with key = seed and counter
 * (row, column, phase, stream); Salmon et al., SC'11. */
typedef struct deco_params {
  int32_t objective;          /* DECO_OBJ_* */
  int32_t precision;          /* DECO_PREC_* storage of the iterate */
  int32_t init;               /* DECO_INIT_* of the first phase */
  int32_t polish_steps;       /* BF16 only: last k steps of every phase in FP32 */
  float eta;                  /* exploration variance (paper: 0.8) */
  float scale;                /* down-scaling of Gaussian starts (paper: 1e-4) */
  float beta;                 /* IDI threshold (paper: 0.2) */
  float uniform_half_width;   /* DECO_INIT_UNIFORM half width (1 = full box) */
  int32_t kernel;             /* DECO_KERNEL_* selector, modifiers included */
  int32_t local_search;       /* deco_solve: at most this many rounds of the
                                 1-flip local search (deco_local_search) on every
                                 phase's rounded vectors before their cuts are
                                 evaluated; 0 = off (the paper's method).  Not
                                 available in deco_solve_batch. */
  int32_t phase_init;         /* deco_solve, phases after the first:
                                 DECO_PHASE_INIT_BEST (0, Sec. 4.2): Gaussian
                                 starts around 2 z* - 1 of the previous phase's
                                 best vector; DECO_PHASE_INIT_FRESH (1): a fresh
                                 start of the first phase's kind (init), its
                                 random draws with the phase index in the
                                 counter (not with DECO_INIT_EXPLICIT).  Batches:
                                 0 only. */
  int32_t eval_every;         /* deco_solve: 0 = off; E > 0 also rounds every
                                 start after steps E, 2E, ... < T_k of every
                                 phase (best-so-far tracking for time-to-target):
                                 these cuts count toward best_cut / best_init /
                                 best_phase / the assignment (ties: the earlier
                                 evaluation); phase_cuts and the next phase's
                                 centre stay the final roundings'.  Batches: 0
                                 only. */
} deco_params;

#define DECO_PHASE_INIT_BEST 0
#define DECO_PHASE_INIT_FRESH 1

int deco_init_block(const deco_graph* g, int32_t B, int32_t lift, int32_t ld,
                    const deco_params* p, uint64_t seed, int32_t phase,
                    const float* mean, const float* x0, void* y, void* stream);

/* IDI mean h_IDI in {-1,+1}^n (Sec. 4.1.2) into device h (n floats). */
int deco_idi_mean(const deco_graph* g, float beta, uint64_t seed, int32_t phase, float* h,
                  void* stream);

/* DUI mean h_DUI (Eq. 12) into device h (n floats). */
int deco_dui_mean(const deco_graph* g, uint64_t seed, int32_t phase, float* h, void* stream);

/* One phase of Alg. 3: lift l = 1 (pQUCO, Alg. 1) or l >= 2 (pLUCO, Alg. 2). */
typedef struct deco_phase {
  int32_t lift;
  int32_t steps;
  float alpha;
  float momentum;
} deco_phase;

typedef struct deco_result {
  int64_t best_cut;       /* best cut over all phases (Alg. 1-3 return value) */
  int32_t best_init;      /* starting point that produced it */
  int32_t best_phase;     /* phase that produced it (earliest on ties) */
  int64_t edge_updates;   /* sum over phases of nnz * B * l * steps */
  double device_ms;       /* device time of the whole solve (CUDA events) */
  int64_t kernel_launches;/* CUDA kernels this solve launched */
} deco_result;

/* pDECO (Alg. 3) over an explicit phase schedule; a one-phase schedule is
 * pQUCO (Alg. 1) or pLUCO (Alg. 2).
 *  B           starting points (>= 1).
 *  phases      host, n_phases entries (1 <= n_phases <= 64).
 *  p           host parameters.
 *  x0          DECO_INIT_EXPLICIT: n x (B*lift0) floats, host or device;
 *              otherwise NULL.
 *  mean        DECO_INIT_MEAN: n floats, host or device; otherwise NULL.
 *  assignment  host, n bytes or NULL: best binary vector (z_v = 1 -> v in S).
 *  phase_cuts  host, n_phases x B int64 or NULL: every starting point's cut
 *              after every phase.
 *  out         host result.
 * Synchronous (one stream sync at the end).  Scratch memory is allocated on
 * the device for the call and released before returning.
 * Errors: DECO_ERR_ARG, DECO_ERR_OOM, DECO_ERR_CUDA, DECO_ERR_NONFINITE. */
int deco_solve(const deco_graph* g, int32_t B, const deco_phase* phases, int32_t n_phases,
               const deco_params* p, uint64_t seed, const float* x0, const float* mean,
               uint8_t* assignment, int64_t* phase_cuts, void* stream, deco_result* out);

/* pDECO under a time budget (Alg. 3: the schedule is repeated while the
 * budget lasts), resumable.  Repetition r runs deco_solve with seed
 * + r; repetition 0 starts as p->init says, or, when `warm` is given, from
 * Gaussian starts around 2 warm - 1; every later repetition starts around
 * 2 z* - 1 of the best vector found so far (DECO_INIT_MEAN, Sec. 4.2).  The
 * call returns after the first repetition whose end brings the summed device
 * time to budget_ms or more, or after max_repeats repetitions.
 *  budget_ms    >= 0 (0: one repetition).
 *  max_repeats  >= 1.
 *  warm         host, n bytes 0/1, or NULL: resume from this assignment (the
 *               assignment of an earlier call); its cut is the best so far.
 *  assignment   host, n bytes or NULL: the best assignment found.
 *  repeats      host int32 or NULL: repetitions run.
 *  out          best cut over the warm start and all repetitions (best_init /
 *               best_phase of the repetition that found it, -1 if the warm
 *               start stayed best); edge_updates, device_ms and
 *               kernel_launches summed over the repetitions.
 * Synchronous.  Errors: as deco_solve. */
int deco_solve_budget(const deco_graph* g, int32_t B, const deco_phase* phases, int32_t n_phases,
                      const deco_params* p, uint64_t seed, double budget_ms, int32_t max_repeats,
                      const uint8_t* warm, uint8_t* assignment, int32_t* repeats, void* stream,
                      deco_result* out);

/* ---------------------------------------------------------------- batches
 * Many graphs solved together with the evolution-based hyper-parameter
 * search of Sec. 4.3.  A batch is the disjoint union of its graphs (a
 * block-diagonal adjacency), so every step kernel runs over all of them in
 * the same launches; rounding, cuts, argmax and best records stay per graph. */
typedef struct deco_batch deco_batch;

/* Build a batch from existing graphs (copied; the graphs may be destroyed
 * afterwards).  Errors: DECO_ERR_ARG, DECO_ERR_OOM, DECO_ERR_CUDA. */
int deco_create_batch(const deco_graph* const* graphs, int32_t n_graphs, deco_batch** out);
void deco_destroy_batch(deco_batch* b);
/* The union graph of a batch (owned by the batch), e.g. for deco_autotune. */
int deco_batch_graph(const deco_batch* b, const deco_graph** out);

/* Population of Sec. 4.3, shared by every graph of the batch.
 *  candidates  P; candidate k owns starts [k B/P, (k+1) B/P) of every graph.
 *  rounds      evolution rounds; round r runs one phase with lift
 *              lifts[r % n_lifts] (e.g. {1, 2}: the pDECO alternation).
 *  t_lo, t_hi  step budgets: T ~ U{t_lo..t_hi}, T' clipped to [t_lo, t_hi].
 *  e_lo, e_hi  alpha = 10^e, e ~ U[e_lo, e_hi], e' = Proj[e_lo, e_hi](e + 0.2 N(0,1)).
 * Candidate k's score is the sum over graphs of the best cut among its
 * starts; after every round the top half is kept (ties: lower index) and
 * the j-th worst member is replaced by a perturbed copy of the j-th best. */
typedef struct deco_population {
  int32_t candidates;
  int32_t rounds;
  int32_t t_lo, t_hi;
  float e_lo, e_hi;
  float momentum;
  int32_t n_lifts;
  int32_t lifts[8];
} deco_population;

/* Batched pDECO with population search (Sec. 4.2, 4.3, Alg. 3).
 *  B           starts per graph, a multiple of pop->candidates.
 *  p           objective, precision (no FP32 polish), init (UNIFORM, IDI or
 *              IDI_HALF_UNIFORM; graph i draws with key seed + i), kernel.
 *  best_cuts   host, n_graphs int64: best cut of every graph over all rounds.
 *  assignment  host, sum of n bytes (graphs in batch order) or NULL.
 *  round_cuts  host, rounds x n_graphs x B int64 or NULL.
 *  round_scores host, rounds x P int64 or NULL.
 *  final_e, final_T  host, P entries each or NULL: the last population.
 *  out         best_cut = sum over graphs; edge_updates counts the longest
 *              budget of every round for all columns.
 * Rounds after the first of a lift replay a captured CUDA graph.  One host
 * synchronisation per round (the evolution runs on the host, in FP64).
 * Errors: DECO_ERR_ARG, DECO_ERR_UNSUPPORTED, DECO_ERR_OOM, DECO_ERR_CUDA,
 * DECO_ERR_NONFINITE, DECO_ERR_TIMEOUT. */
int deco_solve_batch(const deco_batch* b, int32_t B, const deco_params* p, const deco_population* pop,
                     uint64_t seed, int64_t* best_cuts, uint8_t* assignment, int64_t* round_cuts,
                     int64_t* round_scores, float* final_e, int32_t* final_T, void* stream, deco_result* out);

/* ------------------------------------------------------ learned proposal
 * A small message-passing network whose output h = tanh(o) in (-1,1)^n is
 * used as the mean of the Gaussian starts (DECO_INIT_MEAN; Sec. 4.2 draws the
 * starts around a mean vector, here a learned one instead of h_IDI).  The
 * paper's method needs no training; this proposal is an optional start.
 *   X  = [d/Delta, d/mean(d), 1/sqrt(d+1), five U(-1,1) features] per node
 *        (features drawn with Philox, key feat_seed; graph i of a batch uses
 *        feat_seed + i)
 *   H0 = relu(X W0 + b0);  H_l = relu(H_{l-1} Ws_l + (D^-1 A H_{l-1}) Wn_l + b_l)
 *   o  = H_L wo + bo;      loss per graph = min over (z, 1-z) of the mean
 *        logistic loss softplus(-(2z-1) o); batch loss = mean over graphs.
 * Parameters: one flat FP32 vector (W0, b0, [Ws, Wn, b] per layer, wo, bo),
 * Xavier-uniform initialised from Philox (key seed). */
typedef struct deco_mpnn deco_mpnn;

int deco_mpnn_create(int32_t hidden, int32_t layers, uint64_t seed, deco_mpnn** out);
void deco_mpnn_destroy(deco_mpnn* m);
int deco_mpnn_num_params(const deco_mpnn* m, int64_t* count);
/* host copies of the parameters; set also resets the Adam state */
int deco_mpnn_get_params(const deco_mpnn* m, float* host, int64_t count);
int deco_mpnn_set_params(deco_mpnn* m, const float* host, int64_t count);

/* h (device, n floats) = tanh(o) for a graph, or for the union of a batch
 * (exactly one of g and b non-NULL).  precision DECO_PREC_BF16 rounds the
 * hidden activations to bfloat16 between layers. */
int deco_mpnn_infer(const deco_mpnn* m, const deco_graph* g, const deco_batch* b, uint64_t feat_seed,
                    int32_t precision, float* h, void* stream);

/* Loss (host, FP64) and gradient (device, num_params floats, or NULL) for
 * labels z (device, n bytes 0/1: the best assignments the solver found). */
int deco_mpnn_loss_grad(const deco_mpnn* m, const deco_graph* g, const deco_batch* b, const uint8_t* z,
                        uint64_t feat_seed, double* loss, float* grad, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias corrected) on the
 * loss above; `loss` (host, or NULL) receives the loss before the step. */
int deco_mpnn_train_step(deco_mpnn* m, const deco_graph* g, const deco_batch* b, const uint8_t* z,
                         uint64_t feat_seed, float lr, double* loss, void* stream);

/* `steps` Adam steps; losses (host, steps doubles, or NULL) receives the loss
 * before every step (one copy after the last step). */
int deco_mpnn_train(deco_mpnn* m, const deco_graph* g, const deco_batch* b, const uint8_t* z,
                    uint64_t feat_seed, float lr, int32_t steps, double* losses, void* stream);

/* ---------------------------------------------------------------------
 * Greedy comparator and 1-flip local search
 * ------------------------------------------------------------------- */

/* The greedy MaxCut algorithm the paper compares against (App. C.1): fix a
 * vertex ordering, put the first vertex in S and every later vertex on the
 * side that cuts more edges to the vertices already placed (ties: S).  Runs
 * b = 0 .. B-1 in parallel, run b on the random ordering pi_b of [0, n): a
 * balanced 4-round Feistel network on [0, 4^h) (4^h >= n, h >= 1) with round
 * function word 0 of Philox4x32-10 counter (R, b, round, 6), key seed, and
 * cycle walking onto [0, n).
 *  z     device, n x B bytes row-major (z[v*B + b]), receives run b's sides
 *        (1 = S).
 *  cuts  device, B int64, receives every run's cut (Eq. 1).
 * Stream-ordered, asynchronous (scratch: n x B int32 orderings).
 * Errors: DECO_ERR_ARG, DECO_ERR_UNSUPPORTED (n >= 2^30), DECO_ERR_OOM, CUDA. */
int deco_greedy(const deco_graph* g, int32_t B, uint64_t seed, uint8_t* z, int64_t* cuts, void* stream);

/* 1-flip local search on B binary columns, in place.  A round computes the
 * cut change of flipping each node alone, gain_v = sum_u w_vu s_u s_v
 * (s = 1 - 2z), and flips every node whose gain is positive and larger than
 * the gain of each neighbour with a positive gain (equal gains: the lower
 * index wins); those nodes are pairwise non-adjacent, so every round raises
 * the cut by the sum of their gains.  The search stops at a 1-flip local
 * optimum (the binary fixed points of the multilinear step) or after
 * max_rounds rounds.  No counterpart in the paper: a polish of the rounded
 * vectors (deco_params.local_search applies it inside deco_solve).
 *  z           device, n x B bytes row-major, 0/1; updated in place.
 *  max_rounds  >= 0.
 *  cuts        device, B int64, or NULL: the cuts after the search.
 *  rounds      host int32 or NULL: the rounds that flipped at least one node
 *              (when given, the call synchronises the stream).
 * Errors: DECO_ERR_ARG, DECO_ERR_OOM, CUDA. */
int deco_local_search(const deco_graph* g, int32_t B, uint8_t* z, int32_t max_rounds, int64_t* cuts,
                      int32_t* rounds, void* stream);

/* ---------------------------------------------------------------------
 * Diagnostics
 * ------------------------------------------------------------------- */

/* Tensor-core instruction rate of this GPU, the bound of the dense kernels'
 * contraction: one CTA per SM, in which `issuers` threads (1 or 2, each in
 * its own warp) issue `count` tcgen05.mma instructions each (kind::f16,
 * M = 128, N = n in {64, 128, 256}, K = 16, BF16 zeros in shared memory,
 * FP32 accumulators in tensor memory), back to back.  ns_per_instruction
 * (host) receives the mean over SMs of the slowest issuer's time from the
 * first issue to the completion of its last instruction, divided by the
 * SM's instructions (count x issuers): 2 * 128 * n * 16 / ns_per_instruction
 * is the SM's FLOP rate in GFLOP/s.  Synchronises the stream.
 * Errors: DECO_ERR_ARG, DECO_ERR_TIMEOUT (a wait gave up, 1 s), CUDA. */
int deco_probe_mma_rate(int32_t n, int32_t issuers, int32_t count, float* ns_per_instruction, void* stream);

/* Diagnostic: the shared-memory load bandwidth of the GPU, the ceiling of the
 * on-chip kernel's gathers (no paper counterpart).  One CTA of 1024 threads
 * per SM reads `width`-byte words (8 or 16) of a 128 KB shared-memory buffer,
 * a warp's 32 lanes on consecutive words (no bank conflicts), `iters` words
 * per thread (a multiple of 8, at most 2^24).  gbs (host) receives the bytes
 * read by all SMs divided by the launch's duration (CUDA events, after an
 * untimed warm-up launch), in GB/s.  Synchronises the stream.
 * Errors: DECO_ERR_ARG, DECO_ERR_OOM, CUDA. */
int deco_probe_smem_rate(int32_t width, int32_t iters, float* gbs, void* stream);

/* Failure detection of the bounded device waits.  Every spin-wait of the
 * kernels (the on-chip kernel's exchange wait, the dense kernels' mbarrier
 * waits and grid barrier) gives up after 2 s, sets bit 1 of the call's error
 * flag and lets the kernel return, so that a solve reports DECO_ERR_TIMEOUT
 * and the CUDA context stays usable.  This probe runs one of those waits, in a
 * one-thread kernel, on something nothing ever completes:
 *   which 0  the dense kernels' mbarrier wait (an mbarrier nobody arrives at)
 *   which 1  the dense phase kernel's grid barrier (a counter nobody increments)
 *   which 2  the on-chip kernel's exchange wait (an mbarrier nobody arrives at)
 * waited_ms (host, or NULL) receives the kernel's duration (CUDA events).
 * Returns DECO_ERR_TIMEOUT when the wait gave up (the expected outcome; the
 * message gives the time), DECO_OK if it did not.  No paper counterpart.
 * Synchronises the stream.  Errors: DECO_ERR_ARG, DECO_ERR_OOM, CUDA. */
int deco_probe_wait_timeout(int32_t which, float* waited_ms, void* stream);

/* Host-side fault injection for tests of the error paths: the k-th scratch
 * allocation after this call (k >= 1; the stream-ordered temporary buffers
 * that deco_solve, deco_solve_batch, deco_round_cut and the other calls take
 * for one call) fails with DECO_ERR_OOM, as a failed cudaMallocAsync would;
 * the calls must release what they took and leave graphs, batches and the
 * CUDA context usable.  k = 0 disarms it.  Process-wide, not thread-safe
 * against concurrent calls.  No paper counterpart.  Errors: DECO_ERR_ARG. */
int deco_debug_fail_scratch_alloc(int32_t k);

/* Diagnostic for tests of allocation behaviour: the current device's current
 * stream-ordered memory pool, from which every scratch buffer of the library
 * is taken (cudaMallocAsync).  used_now (host, or NULL) receives the bytes of
 * the pool in use now, used_high (host, or NULL) the most bytes in use at once
 * since the high-water mark was last reset; reset != 0 then restarts the
 * high-water mark from the current use.  Process-wide (the pool is shared with
 * every other user of it in the process).  No paper counterpart.
 * Errors: CUDA. */
int deco_debug_pool_usage(int64_t* used_now, int64_t* used_high, int32_t reset);

/* Thread-local message of the last error on this thread ("" if none). */
const char* deco_last_error(void);

/* ABI version (DECO_ABI_VERSION) of the loaded library. */
int deco_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DECO_H_ */
