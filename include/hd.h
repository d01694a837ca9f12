/*
 * hd.h -- C ABI of the GB300 one-step overlapping DDM Helmholtz solver.
 *
 * Method: Leng & Ju, "An overlapping domain decomposition preconditioner for
 * the Helmholtz equation" (arXiv 1508.02897).  The 2D Helmholtz problem
 * Delta u + k^2 u = f (Eq. (helm)) is truncated by a uniaxial PML (Sec. 2,
 * Eq. (pml)) and discretised by a conservative second-order 5-point stencil
 * (Sec. 3).  GMRES (Sec. 3) is preconditioned by the one-step DDM
 * preconditioner of Eq. (ddm0) and Eq. (pc): restrict the residual to every
 * owned box, solve every local PML problem of Eq. (pmlij) at once, and add
 * every full local solution, including its PML area, back into the global
 * vector.
 *
 * Conventions shared by every entry point
 *  - Every function returns an hd_status (HD_OK = 0); hd_last_error() gives a
 *    message for the calling thread.  No C++ exception crosses this boundary.
 *  - Grid: interior nx x ny cells of width h plus npml PML cells on every side;
 *    the global grid is NX = nx + 2 npml by NY = ny + 2 npml, stored row by row
 *    (x fastest).  A complex vector is interleaved double re/im
 *    (C99 double _Complex / numpy complex128) of NX*NY entries per right-hand
 *    side; several right-hand sides are stored one after another.
 *  - Pointers named *_dev are device pointers owned by the caller; the library
 *    never frees them.  Workspaces are sized by hd_query_workspace and allocated
 *    by the caller (for instance with torch.empty on the device).
 *  - `stream` is a cudaStream_t passed as void*.  Calls are asynchronous on it
 *    unless stated otherwise.
 *  - A context is not thread safe: one host thread per context at a time.
 */
#ifndef HD_H_
#define HD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HD_OK = 0,
  HD_ERR_INVALID = 1,        /* bad argument, size or state                      */
  HD_ERR_OOM = 2,            /* a workspace is too small / allocation failed     */
  HD_ERR_CUDA = 3,           /* a CUDA runtime call failed                        */
  HD_ERR_NOT_CONVERGED = 4,  /* GMRES hit max_iters (stats are still filled in)   */
  HD_ERR_NUMERIC = 5,        /* NaN/Inf or a zero pivot                           */
  HD_ERR_TIMEOUT = 6,        /* a bounded device wait gave up                      */
  HD_PENDING = 7             /* reserved for asynchronous request handles          */
} hd_status;

typedef enum {
  HD_C128 = 0,  /* local factors and substitutions in complex FP64              */
  HD_C64 = 1,   /* local factors and substitutions in complex FP32, FP64 outside */
  HD_C64_H = 2, /* as HD_C64, but the stored S_j^{-1} are complex FP16 (half the
                   bytes streamed by every preconditioner application); the
                   factorisation recursion itself stays FP32                     */
  HD_C64_B = 3  /* as HD_C64_H with complex BF16 storage: the same halved bytes,
                   an 8-bit mantissa instead of 11 but FP32's exponent range     */
} hd_precision;

/* Flag OR-ed into the precision of hd_setup_medium: store only the upper
 * 16 x 16 tiles of every S_j^{-1} (which is complex symmetric, because the
 * operator is), so each preconditioner application streams about 55% of the
 * bytes; the stored inverse is the exactly symmetric matrix built from the
 * computed inverse's upper triangle. */
#define HD_SYMMETRIC 0x100

/* Flag OR-ed into HD_C64 (not with HD_SYMMETRIC): store every S_j^{-1} rounded to
 * TF32 as real and imaginary planes in the operand layout of the tensor cores, and
 * run each substitution step Y = S_j^{-1} V for groups of 16 right-hand sides as
 * tcgen05 TF32 MMAs with FP32 accumulation ([Yr | Yi] = Sr [Vr | Vi] + Si [-Vi | Vr]).
 * Meant for many sources sharing one medium (the factor is read once per group of
 * 16 instead of once per 8); storage is m rounded up to 8, squared, 8 bytes per
 * entry.  The factorisation itself stays FP32; only the stored copy is TF32. */
#define HD_TCORE 0x200

/* Flag OR-ed into HD_C64 | HD_TCORE: keep FP32-grade products on the tensor cores.
 * Every stored entry x of S_j^{-1} becomes a pair of TF32 numbers (x_hi = x rounded
 * to TF32, x_lo = the rest rounded to TF32, |x - x_hi - x_lo| <= 2^-22 |x|), the
 * right-hand sides are split the same way, and each substitution step takes the
 * products hi*hi + lo*hi + hi*lo (+ lo*lo) with FP32 accumulation, for groups of 32
 * right-hand sides per CTA: the accuracy of the FP32 substitution at the factor bytes
 * per right-hand side of the TF32 storage (16 bytes per entry, read once per 32).
 * Boxes up to 176 cells wide (hd_setup_medium returns HD_ERR_INVALID otherwise). */
#define HD_TF32X3 0x800

/* Flag OR-ed into any precision: weight every local solution by the smoothing
 * function beta_ij of the Remark after Eq. (pc) before the sum of Eq. (pc)
 * (beta = 1 on the owned cells, a C^2 step t^3 (10 - 15 t + 6 t^2) of the distance
 * across the overlap + PML band, 0 just past the box; the paper states the
 * properties, not the profile).  Applies to the one-step preconditioner, and
 * hd_apply_ddm then does residual correction with this smoothed M. */
#define HD_SMOOTH 0x400

/* Truncated domain Omega of Sec. 2: interior nx x ny cells of width h (the
 * interior is [0, nx h] x [0, ny h]), npml PML cells per side.  The PML uses
 * alpha(xi) = 1 + i sigma(xi)/omega with sigma(xi)/omega =
 * sigma0_over_omega * (xi / (npml h))^pml_power, xi the distance into the layer. */
typedef struct {
  int32_t nx, ny, npml;
  double h;
  double omega;
  double sigma0_over_omega;
  int32_t pml_power;
} hd_grid;

/* Decomposition of Sec. 2 (Fig. 1): nbx x nby owned boxes cut at the interior
 * cut points cut_x[0..nbx] (cut_x[0] = npml, cut_x[nbx] = npml + nx; NULL =
 * even cuts), likewise cut_y; each box is extended by `overlap` cells (lo) plus
 * npml local PML cells on its inner sides and by npml cells on its outer sides.
 * own_global_pml = 1 lets the boundary boxes also own the adjacent global-PML
 * cells so the owned boxes tile the whole grid; 0 is the literal reading
 * (owned boxes tile the interior only).  Every owned width must be at least
 * overlap + npml.  The arrays are copied; the caller keeps ownership. */
typedef struct {
  int32_t nbx, nby, overlap;
  const int32_t *cut_x;
  const int32_t *cut_y;
  int32_t own_global_pml;
} hd_decomp;

typedef struct hd_ctx hd_ctx;

/* Creates a context for one medium (Sec. 2, Eq. (pml)): copies the grid and
 * decomposition, computes k^2 = (omega / c)^2 on the device from the velocity
 * c_dev (FP64, NY x NX, device memory, read during the call only), the global
 * and per-box PML stretching tables and the box tables.  Allocates its own
 * device tables (about 8 NX NY bytes plus O(boxes)) stream-ordered on `stream`
 * (cudaMallocAsync); synchronises `stream` before returning.  On error *out is
 * NULL. */
int hd_setup_medium(hd_ctx **out, const hd_grid *grid, const hd_decomp *decomp, const double *c_dev,
                    int32_t precision, void *stream);

/* Bytes the caller must provide:
 *   factor_bytes  : the per-box Schur inverses written by hd_factor_subdomains
 *   krylov_bytes  : FGMRES bases V (restart+1 vectors) and Z (restart vectors),
 *                   two work vectors and the Hessenberg/reduction scratch, for
 *                   nrhs right-hand sides solved together
 *   scratch_bytes : per-box staging of the local substitutions for nrhs
 *                   right-hand sides (apply) or the per-box working matrix
 *                   (factorisation), whichever is larger
 * Any output pointer may be NULL.  nrhs >= 1 and 1 <= restart <= HD_MAX_RESTART,
 * else HD_ERR_INVALID. */
int hd_query_workspace(const hd_ctx *ctx, int32_t nrhs, int32_t restart, size_t *factor_bytes,
                       size_t *krylov_bytes, size_t *scratch_bytes);

/* Factorises every local PML problem of Eq. (pmlij) (Sec. 3: "factorized and
 * solved with direct solver") as a block-tridiagonal LU along the grid rows of
 * the box: S_0 = D_0, S_j = D_j - L_j S_{j-1}^{-1} U_{j-1} (L_j, U_j diagonal,
 * D_j tridiagonal), storing every S_j^{-1} (m x m, m = box width, column-major)
 * in factor_dev.  Each S_j is inverted by Gauss-Jordan elimination.  With
 * complex FP32 arithmetic (HD_C64, HD_C64_H) and boxes at most 192 wide the
 * default kernel keeps S_j in tensor memory and eliminates it without pivoting,
 * 16 columns per step, each step one rank-16 complex update on the tensor cores
 * (tcgen05 MMAs on operands split into three BF16 pieces, FP32 accumulation);
 * it checks every pivot, and a box with a pivot below pivot_ratio times the
 * largest unprocessed entry of its column (hd_set_factor_path) is factorised
 * again by the SIMT kernel with partial pivoting, in the same call.  Otherwise
 * (HD_C128, wider boxes, or HD_FACTOR_SIMT) the SIMT kernel with partial
 * pivoting factorises every box.  factor_dev stays bound to the context (the
 * caller keeps it alive until hd_destroy or the next factorisation).
 * scratch_dev is free again when the call's work on `stream` ends.  Returns
 * HD_ERR_NUMERIC later (from hd_gmres_solve / hd_check_status) if a pivot was
 * zero. */
int hd_factor_subdomains(hd_ctx *ctx, void *factor_dev, size_t factor_bytes, void *scratch_dev,
                         size_t scratch_bytes, void *stream);

/* Kernel choice of hd_factor_subdomains (no counterpart in the paper, which names
 * no direct solver). */
typedef enum {
  HD_FACTOR_AUTO = 0,   /* tensor cores where they apply, else the SIMT kernel          */
  HD_FACTOR_SIMT = 1,   /* Gauss-Jordan with partial pivoting on the CUDA cores         */
  HD_FACTOR_TCORE = 2   /* tensor cores; hd_factor_subdomains fails with HD_ERR_INVALID
                           where they do not apply                                     */
} hd_factor_path;

/* Selects the factorisation kernel for later hd_factor_subdomains calls on ctx and
 * the pivot check of the tensor-core kernel: a box is refactorised with partial
 * pivoting when some pivot p has |p| < pivot_ratio * max |entry| over the other
 * unprocessed rows checked in its column (0 < pivot_ratio; the default 0.5 lets
 * multipliers reach at most 2).  HD_ERR_INVALID for an unknown path or a
 * non-positive or non-finite ratio. */
int hd_set_factor_path(hd_ctx *ctx, int32_t path, double pivot_ratio);

/* How the last hd_factor_subdomains on ctx factorised its boxes: *tcore_boxes
 * kept the tensor-core result, *pivoted_boxes were (re)factorised with partial
 * pivoting.  Synchronises `stream`.  Outputs may be NULL; HD_ERR_INVALID before
 * any factorisation. */
int hd_factor_report(hd_ctx *ctx, int32_t *tcore_boxes, int32_t *pivoted_boxes, void *stream);

/* y = A x for nrhs vectors: A is the PML operator of Eq. (pml) multiplied by
 * J h^2 (J = alpha1 alpha2), a complex-symmetric 5-point matrix with
 * homogeneous Dirichlet values outside Omega.  x_dev, y_dev: complex128
 * [nrhs][NY][NX], must not overlap. */
int hd_matvec(hd_ctx *ctx, const void *x_dev, void *y_dev, int32_t nrhs, void *stream);

/* b = J h^2 f: the right-hand side of the scaled system for source samples f
 * (complex128 [nrhs][NY][NX]); b may equal f. */
int hd_rhs_from_source(hd_ctx *ctx, const void *f_dev, void *b_dev, int32_t nrhs, void *stream);

/* z = sum_ij E_ij^T A_ij^{-1} X_ij r, Eq. (ddm0) + Eq. (pc): X_ij restricts r to
 * the owned box, A_ij is the local PML operator of Eq. (pmlij) on the
 * overlapping box (solved with the stored factors), E_ij^T extends the local
 * solution over the whole box, PML area included, and the sum runs in a fixed
 * order (deterministic).  r_dev, z_dev: complex128 [nrhs][NY][NX], must not
 * overlap.  Needs a prior hd_factor_subdomains.  scratch_dev: at least
 * scratch_bytes of hd_query_workspace for nrhs = 1; with room for g right-hand
 * sides they are processed g at a time, each factor block read once per group
 * (up to 8 right-hand sides per CTA). */
int hd_apply_precond(hd_ctx *ctx, const void *r_dev, void *z_dev, int32_t nrhs, void *scratch_dev,
                     size_t scratch_bytes, void *stream);

/* Multi-step overlapping DDM, Eq. (ddm0), (ddms) and (sum): u = the sum over
 * steps s < nsteps of every box's local solution, step 0 with f restricted to the
 * owned boxes, step s+1 with minus the sum of the neighbours' L u^s restricted to
 * them (L: the operator of the whole truncated domain).  Since a box's own
 * residual vanishes on its owned part (Sec. 2), the step-(s+1) sources are the
 * global residual of the sum so far, and this is computed as
 *     u_0 = M f,   u_{s+1} = u_s + M (f - A u_s),   M = hd_apply_precond.
 * nsteps = 1 is hd_apply_precond.  f_dev, u_dev: complex128 [nrhs][NY][NX], u is
 * the output and must not alias f; work_dev: 2 * nrhs * NX * NY * 16 bytes (the
 * residual and the correction); scratch as for hd_apply_precond (nrhs vectors
 * at once).  Asynchronous on stream. */
int hd_apply_ddm(hd_ctx *ctx, const void *f_dev, void *u_dev, int32_t nrhs, int32_t nsteps, void *work_dev,
                 size_t work_bytes, void *scratch_dev, size_t scratch_bytes, void *stream);

/* Arithmetic of the Gram-Schmidt dot products and updates. */
typedef enum {
  HD_ARNOLDI_FP64 = 0,  /* IEEE FP64 throughout                                       */
  HD_ARNOLDI_DS = 1     /* basis stored as float pairs (hi + lo, ~48-bit mantissa) and
                           double-single arithmetic on the FP32 pipes; norms, Givens,
                           least squares and the true residual stay FP64               */
} hd_arnoldi_mode;

/* Preconditioner application that allocates nothing.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc
 * when they apply the preconditioner (plug-ins whose host application owns the
 * device heap, latency-bound loops where an allocation could synchronise the
 * device, services that must keep a fixed device footprint after start-up).
 * Same result as hd_apply_precond, but the staging vectors live in a fixed
 * 64 MiB device array inside the library instead of a caller workspace; every
 * GPU that loads the library holds that array until the process exits.  The
 * first call in a CUDA context (device and driver context, primary or made by
 * the caller) looks up the array's device address there (cudaGetSymbolAddress)
 * and remembers it for that context; make that first call before any stream
 * capture.  A context destroyed by cudaDeviceReset whose replacement happens to
 * get the same driver handle is not told apart, so after a reset make the next
 * call through a fresh process or context.  A problem whose staging vectors need more than 64 MiB
 * (scratch_bytes of hd_query_workspace for the substitution) is refused with
 * HD_ERR_OOM.  Every call shares the one array and it keeps the last call's
 * contents (no entry is read before the same call writes it, so nothing needs
 * clearing); calls whose work overlaps on the GPU -- other streams, contexts or
 * threads -- race on it, so the caller must serialise them.  r_dev, z_dev as in
 * hd_apply_precond; right-hand sides are processed in groups that fit the array. */
int hd_apply_precond_noalloc(hd_ctx *ctx, const void *r_dev, void *z_dev, int32_t nrhs, void *stream);

/* Largest FGMRES restart length (Krylov vectors per cycle) the solver takes; the
 * per-step Gram-Schmidt kernels keep one coefficient per basis vector in shared
 * memory. */
#define HD_MAX_RESTART 256

typedef struct {
  int32_t restart;    /* Krylov vectors per cycle, 1 .. HD_MAX_RESTART              */
  int32_t max_iters;  /* Arnoldi steps over all cycles                             */
  double rtol;        /* stop when ||b - A x|| <= rtol ||b||                        */
  int32_t use_x0;     /* 1: start from x_dev, 0: x0 = 0                              */
  int32_t arnoldi;    /* hd_arnoldi_mode                                            */
  int32_t graphs;     /* 1: capture each Arnoldi step j (preconditioner, matvec, CGS2,
                         Givens, normalisation) once as a CUDA graph per workspace and
                         replay it in later cycles and solves; 0: plain launches   */
  int32_t reorth;     /* 0: always two Gram-Schmidt passes (CGS2); 1: second pass only
                         when the first cancelled more than a factor 10 of ||w||
                         (Rutishauser's criterion, decided on the device)          */
  int32_t precond_steps; /* steps of the overlapping DDM used as the preconditioner
                         (hd_apply_ddm); 0 or 1: the one-step preconditioner of
                         Eq. (pc)                                                  */
} hd_gmres_opts;

typedef struct {
  int32_t iters;        /* Arnoldi steps over all cycles                            */
  int32_t restarts;     /* completed cycles                                          */
  int32_t converged;    /* 1 if the true relative residual <= rtol                   */
  int32_t status;       /* hd_status of this right-hand side                         */
  double relres_est;    /* |g_{k}| / ||b|| from the Givens recurrence                */
  double relres_true;   /* ||b - A x|| / ||b|| recomputed in FP64                    */
  double t_solve_s;     /* wall time of the solve on the host                        */
  int32_t second_passes;/* Arnoldi steps that ran the second Gram-Schmidt pass         */
  int32_t second_pass_vecs; /* basis vectors those second passes went over (sum of j+1) */
} hd_gmres_stats;

/* Restarted right-preconditioned flexible GMRES (Sec. 3; Z_j = M v_j stored):
 * classical Gram-Schmidt applied twice (FP64 or double-single, opts->arnoldi),
 * FP64 norms and complex Givens rotations with
 * real cosine, x += Z y at the end of each cycle, and the FP64 true residual
 * b - A x decides convergence.  Blocking: returns when every right-hand side
 * has converged or failed, with stats_host[nrhs] filled in.  b_dev, x_dev:
 * complex128 [nrhs][NY][NX]; x_dev is the output (and the start when use_x0).
 * The nrhs right-hand sides are solved together in lockstep (one independent
 * FGMRES each; every preconditioner launch serves all of them, a converged one
 * stops while the others go on); krylov_dev and scratch_dev must be sized by
 * hd_query_workspace for (nrhs, restart).  Returns HD_ERR_NOT_CONVERGED if any
 * right-hand side missed rtol within max_iters. */
int hd_gmres_solve(hd_ctx *ctx, const void *b_dev, void *x_dev, int32_t nrhs, const hd_gmres_opts *opts,
                   void *krylov_dev, size_t krylov_bytes, void *scratch_dev, size_t scratch_bytes,
                   hd_gmres_stats *stats_host, void *stream);

/* Largest block (right-hand sides sharing one Krylov space) of hd_block_gmres_solve. */
#define HD_MAX_BLOCK 128

/* Bytes of the block solver's workspaces for p right-hand sides and `restart` block
 * steps per cycle: krylov_bytes holds the block bases V ((restart+1) p vectors) and
 * Z (restart p), one more block and the Gram reduction buffers; scratch_bytes the
 * substitution staging of p right-hand sides (or the factorisation working matrix,
 * whichever is larger).  Outputs may be NULL; HD_ERR_INVALID for p outside
 * 1 .. HD_MAX_BLOCK or restart outside 1 .. HD_MAX_RESTART. */
int hd_query_block_workspace(const hd_ctx *ctx, int32_t p, int32_t restart, size_t *krylov_bytes,
                             size_t *scratch_bytes);

/* Block flexible GMRES (Sec. 3's GMRES taken to p sources sharing one Krylov space;
 * the block method of Saad, Iterative Methods for Sparse Linear Systems, Sec. 6.12,
 * flexible as in Sec. 9.4): per cycle R = B - A X = V_0 S (thin QR); block step j
 * applies the one-step preconditioner of Eq. (pc) to the p columns of V_j in one
 * launch (Z_j), W = A Z_j, block classical Gram-Schmidt twice (H_ij = V_i^H W for all
 * i <= j from the same W, W -= sum V_i H_ij), W = V_{j+1} H_{j+1,j} by Cholesky QR done
 * twice; the least squares min || E_1 S - Hbar Y ||_F is updated on the host (FP64
 * Householder QR) and gives each column's residual estimate.  The cycle ends when every
 * estimate is <= rtol, at the restart, or when a new block loses a direction; then
 * X += [Z_0 .. Z_k] Y and the FP64 true residual decides.  All of it runs in FP64 but the
 * preconditioner, which uses the context's precision.  b_dev, x_dev: complex128
 * [p][NY][NX]; x_dev is the output (and the start when opts->use_x0).  opts->restart
 * counts block steps per cycle, opts->max_iters block steps in all; arnoldi, graphs
 * and reorth are ignored, precond_steps must be 0 or 1.  Blocking; stats_host[p]: iters
 * = block steps (each one preconditioner launch for the p columns), converged and
 * relres_true per column.  HD_ERR_NUMERIC if the first residual block is rank deficient
 * (dependent sources: solve them separately), HD_ERR_NOT_CONVERGED if a column missed
 * rtol within max_iters. */
int hd_block_gmres_solve(hd_ctx *ctx, const void *b_dev, void *x_dev, int32_t p, const hd_gmres_opts *opts,
                         void *krylov_dev, size_t krylov_bytes, void *scratch_dev, size_t scratch_bytes,
                         hd_gmres_stats *stats_host, void *stream);

/* Autotuner (no counterpart in the paper): times hd_apply_precond's
 * substitution kernel for each candidate launch shape (96, 128, 192 or 256
 * consumer threads per CTA, 2 to 32 ring stages that fit shared memory) on r_dev ->
 * z_dev (complex128 NY x NX, contents irrelevant, z is overwritten) with CUDA
 * events on `stream`, and keeps the fastest for this context.  The choice is
 * remembered for the process per (precision, storage layout, widest box,
 * number of boxes, device), and hd_setup_medium applies a remembered choice to every
 * later context of the same shape (no timing).  The server tunes the first request of
 * each shape this way.  Needs a prior hd_factor_subdomains; synchronises `stream`.  Any output
 * pointer may be NULL; *ms_out is the winner's time per application (-1 when
 * taken from the cache). */
int hd_autotune(hd_ctx *ctx, const void *r_dev, void *z_dev, void *scratch_dev, size_t scratch_bytes,
                int32_t *threads_out, int32_t *stages_out, float *ms_out, void *stream);

/* Per-kernel-class timing with CUDA events recorded on the launching stream
 * (events only while profiling is on; off by default).  Classes: 0
 * factorisation, 1 restrict + forward/back substitution, 2 gather-sum,
 * 3 matvec/residual, 4 Arnoldi (dots, updates, Givens, solution update),
 * 5 other.  hd_get_timers writes ms[class] (accumulated device time, profiled
 * launches only) and launches[class] (kernels launched, always counted) for up
 * to n classes and synchronises `stream`; reset = 1 clears both afterwards. */
int hd_set_profiling(hd_ctx *ctx, int32_t on);
int hd_get_timers(hd_ctx *ctx, double *ms, int64_t *launches, int32_t n, int32_t reset, void *stream);

/* Reads the device status word (set by kernels on a zero pivot, a non-finite
 * value or a bounded wait that gave up), synchronising `stream`; clear = 1
 * resets it. */
int hd_check_status(hd_ctx *ctx, int32_t clear, void *stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching of solve requests on one GPU (no counterpart in the
 * paper, whose solves ran one at a time on a cluster).  A server owns
 * max_slots worker threads, each with its own non-blocking stream.  A
 * submitted request waits in a first-come-first-served queue until a slot is
 * free and its device memory (context tables, factors, Krylov bases, staging
 * and vectors; all from the stream-ordered allocator, so no allocation
 * synchronises the device) fits in what is left of hbm_budget_bytes; admitted
 * requests run concurrently and their kernels overlap on the device.  Each
 * request keeps its factors and Krylov bases resident until it completes.  A
 * request whose nrhs right-hand sides do not fit the budget together is solved
 * in lockstep sub-batches that do.  Results do not depend on what else runs. */
typedef struct hd_server hd_server;

typedef struct {
  double queue_s;        /* submit -> admission                                      */
  double run_s;          /* admission -> completion                                  */
  double latency_s;      /* submit -> completion                                     */
  uint64_t device_bytes; /* device memory reserved while running                     */
  int32_t batch;         /* right-hand sides per lockstep sub-batch                  */
} hd_request_info;

typedef struct {
  int32_t queued, running, peak_running;
  uint64_t completed, bytes_in_use, peak_bytes_in_use, budget_bytes;
} hd_server_counters;

/* Starts a server on CUDA device `device` with max_slots (1..64) concurrent
 * requests and a device memory budget in bytes.  Requests allocate their device
 * memory from a memory pool of the server's own that keeps up to the budget mapped
 * between requests (released by hd_server_destroy). */
int hd_server_create(hd_server **out, size_t hbm_budget_bytes, int32_t max_slots, int32_t device);

/* Queues one solve: medium c_host (FP64 velocity, NY x NX), sources f_host
 * (complex128 [nrhs][NY][NX], turned into b = J h^2 f on the device), FGMRES
 * options, output x_host (complex128 [nrhs][NY][NX]).  The three host buffers
 * are the caller's and must stay valid until hd_poll returns something other
 * than HD_PENDING for the ticket.  The grid/decomposition structs and cut
 * arrays are copied.  HD_ERR_OOM if one right-hand side alone exceeds the
 * budget. */
int hd_submit(hd_server *srv, const hd_grid *grid, const hd_decomp *decomp, const double *c_host, const void *f_host,
              int32_t nrhs, int32_t precision, const hd_gmres_opts *opts, void *x_host, uint64_t *ticket);

/* Waits up to timeout_us (0: do not wait, < 0: wait forever) for a ticket.
 * HD_PENDING while it is queued or running; otherwise the request's status,
 * with stats[nrhs] and *info (either may be NULL) filled in and the ticket
 * released. */
int hd_poll(hd_server *srv, uint64_t ticket, hd_gmres_stats *stats, hd_request_info *info, int64_t timeout_us);

/* Snapshot of the server's counters. */
int hd_server_info(hd_server *srv, hd_server_counters *out);

/* Stops the server: requests already running finish, queued ones are dropped
 * (their tickets become invalid), the worker threads are joined. */
int hd_server_destroy(hd_server *srv);

/* Frees the context's own device tables (not the caller's workspaces), stream
 * ordered after the work queued on the stream given to hd_setup_medium (which
 * must still exist); does not synchronise the device. */
int hd_destroy(hd_ctx *ctx);

/* Message of the last error on the calling thread ("" if none). */
const char *hd_last_error(void);

/* Library version string. */
const char *hd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HD_H_ */
