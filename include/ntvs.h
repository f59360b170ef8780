/*
 * ntvs.h - C ABI of the GB300 (sm_103a) NTVS reconstruction library.
 *
 * NTVS = total variation superiorization with N normalized TV perturbation steps of
 * size beta0*alpha^ell between feasibility-seeking sweeps, with or without the TV
 * reduction check (arXiv 1803.01112, Sec. III-B, Appendix C).  The feasibility-seeking
 * operator P_T is one sweep of block-DROP over the blocks of proton histories
 * (Sec. III-D, DROP of ref. CEHN08):
 *
 *     for each block t, with every row i of the block seeing the same x:
 *       r_i  = (b_i - <a_i, x>) / ||a_i||^2            (0 when ||a_i|| = 0)
 *       x_j += lambda * (1/s_j^t) * sum_{i in t} a_ij r_i   (only where s_j^t > 0)
 *     s_j^t = number of stored entries (i, j) of block t with a_ij != 0.
 *
 * phi = TV = sum over voxels of the Euclidean length of the forward-difference
 * vector (TV is introduced in Sec. II with ref. CCCNP10), index spacing, difference past the last index = 0.
 * The perturbation direction is v = -grad phi_eps / ||grad phi_eps|| (Appendix A),
 * phi_eps(x) = sum_p sqrt(eps + |forward differences at p|^2); v = 0 if the gradient is 0.
 *
 * Conventions for every entry point:
 *   - returns NTVS_OK (0) or a negative NTVS_ERR_* code; ntvs_last_error() gives the
 *     calling thread's last message.  No C++ exception crosses the ABI.
 *   - images are dense [nz][ny][nx] (x fastest), voxel index (iz*ny + iy)*nx + ix.
 *   - NTVS_MEM_HOST pointers are copied during the call (the caller keeps ownership).
 *     NTVS_MEM_DEVICE pointers must be device memory of the context's GPU; system
 *     arrays passed that way are borrowed and must outlive the context (or the next
 *     ntvs_load_system).  Output buffers are allocated by the caller.
 *   - work is queued on the context's CUDA stream; device-memory outputs are ready
 *     when that stream reaches them, host outputs when the call returns.
 *   - a context is not thread safe: one thread at a time per context.
 */
#ifndef NTVS_H
#define NTVS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NTVS_OK 0
#define NTVS_ERR_ARG (-1)      /* bad argument, size or pointer                       */
#define NTVS_ERR_CSR (-2)      /* malformed system (row_ptr, col range, non-finite)   */
#define NTVS_ERR_OOM (-3)      /* device allocation failed                            */
#define NTVS_ERR_CUDA (-4)     /* a CUDA runtime call or kernel launch failed         */
#define NTVS_ERR_TIMEOUT (-5)  /* a bounded device-side wait ran out                  */
#define NTVS_ERR_STATE (-6)    /* call made in the wrong state (e.g. no system yet)   */

/* element types */
#define NTVS_F64 0
#define NTVS_F32 1
#define NTVS_F16 2
#define NTVS_BF16 3

/* memory kinds */
#define NTVS_MEM_HOST 0
#define NTVS_MEM_DEVICE 1

/* index storage of the system on the device */
#define NTVS_CSR32 0     /* int32 column per entry                                      */
#define NTVS_DELTA16 1   /* 16-bit columns, packed at load time: the entries are cut into
                            aligned chunks of 32; each chunk keeps an int32 base and every
                            entry its uint16 offset from it: the row's smallest column for a
                            row whose columns span at most 65535, else the chunk's smallest
                            column (a chunk whose columns span more than 65535 keeps full
                            int32 columns); 2.125 bytes per entry plus escapes            */

typedef struct ntvs_ctx ntvs_ctx;

/* The linear system of one reconstruction: row i is proton history i, a_ij its
 * intersection length with voxel j, b_i its WEPL (Sec. I, Sec. III-D). */
typedef struct {
    int32_t nx, ny, nz;          /* image grid, V = nx*ny*nz                                */
    int32_t n_blocks;            /* B; used when block_ptr is NULL: contiguous blocks of
                                    ceil(M/B) rows in stored order                           */
    int64_t n_rows;              /* M >= 0                                                    */
    const int64_t* row_ptr;      /* [M+1], row_ptr[0] = 0, non-decreasing (mem_kind)          */
    const int32_t* col;          /* [nnz] voxel index in [0, V) (mem_kind)                    */
    const void* val;             /* [nnz] a_ij, type val_dtype (mem_kind)                     */
    const void* b;               /* [M] WEPL, double if val_dtype == NTVS_F64 else float
                                    (also with ntvs_set_compute_dtype(NTVS_F64))             */
    const int64_t* block_ptr;    /* NULL or [B+1] HOST array, block t = rows [bp[t], bp[t+1]) */
    int32_t val_dtype;           /* NTVS_F64 (FP64 path) | NTVS_F32 (FP32 path) |
                                    NTVS_F16 / NTVS_BF16 (FP32 arithmetic on half storage)   */
    int32_t mem_kind;            /* NTVS_MEM_HOST | NTVS_MEM_DEVICE (row_ptr, col, val, b)    */
    int32_t storage;             /* NTVS_CSR32 | NTVS_DELTA16                                 */
    int32_t schedule;            /* DROP kernel schedule: NTVS_SCHED_AUTO (0), NTVS_SCHED_PLAIN,
                                    NTVS_SCHED_WINDOW (see below)                             */
} ntvs_system;

/* DROP kernel schedules.  PLAIN: rows in stored order, every scatter a global reduction.
 * WINDOW: rows grouped at load time by their home z-slice (median slice of the rows of
 * each 64-row chunk); one CTA per SM accumulates its slice in shared memory (needs
 * nx*ny*sizeof(compute type) of shared memory per CTA).  PIPELINE: WINDOW's grouping
 * with the matrix streamed into shared memory by the TMA engine (cp.async.bulk) ahead of
 * the consumer warps; needs 16-byte aligned col/val and 64 KB more shared memory.  When
 * the slice fits and rows come in runs of the same slice (e.g. stored by projection angle,
 * then slice), AUTO picks WINDOW (measured fastest); otherwise PLAIN.  Every schedule reads
 * both index storages.  All give the same result up to the order of floating-point
 * summation. */
#define NTVS_SCHED_AUTO 0
#define NTVS_SCHED_PLAIN 1
#define NTVS_SCHED_WINDOW 2
#define NTVS_SCHED_PIPELINE 3
#define NTVS_SCHED_ONTHEFLY 4   /* reported for systems loaded with ntvs_load_paths */

/* Step-size rules of the TV perturbations (ntvs_params.step_rule). */
#define NTVS_STEP_NTVS 0       /* ell_k = rand(k, ell_{k-1}); try t of cycle k uses
                                  beta0 * alpha^(ell_k + t) (Appendix C)                      */
#define NTVS_STEP_OTVS 1       /* ell never reset: ell_k = ell_{k-1} (Appendix B); the paper's
                                  OTVS is this rule with N = 1, alpha = 1/2, beta0 = 1 and
                                  tv_check = 1                                                */
#define NTVS_STEP_DECOUPLED 2  /* beta_{k,n} = beta0 * alpha^n * gamma^k, n = 0..N-1, k the
                                  cycle index from 0 (Sec. VI); no ell, no TV check           */

/* Parameters of NTVS (Sec. III-E, Appendix A/C). */
typedef struct {
    double lambda;       /* DROP relaxation lambda                                        */
    double alpha;        /* perturbation kernel, 0 < alpha < 1                             */
    double beta0;        /* beta_{k,n} = beta0 * alpha^ell; the paper's value is 1         */
    double eps_tv;       /* epsilon of phi_eps in the gradient (>= 0; default 1e-8)        */
    int32_t N;           /* TV perturbation steps per cycle, >= 0                          */
    int32_t tv_check;    /* 0: NTVS; 1: NTVS with the TV reduction requirement             */
    int32_t max_retries; /* tries per step in check mode before the step is skipped (>=1) */
    int32_t step_rule;   /* NTVS_STEP_NTVS (0), NTVS_STEP_OTVS or NTVS_STEP_DECOUPLED       */
    uint64_t seed;       /* stream of the ell draws (SplitMix64, output k for cycle k)     */
    double gamma;        /* decoupled rule only: 0 < gamma < 1                             */
} ntvs_params;

typedef struct {
    int64_t k;             /* cycles completed                                           */
    int64_t ell_prev;      /* ell_{k-1}, the exponent carried into the next cycle        */
    int64_t n_steps;       /* perturbation steps taken (N per cycle)                     */
    int64_t n_accepted;    /* steps that changed x                                       */
    int64_t n_tries;       /* tries (check mode: >= n_steps)                             */
    int64_t nnz;           /* stored entries of the loaded system                        */
    int64_t n_rows;        /* M                                                          */
    int32_t n_blocks;      /* B                                                          */
    int32_t compute_dtype; /* NTVS_F64 or NTVS_F32                                       */
    double last_tv;        /* phi(x) after the last completed cycle (FP64)               */
    int64_t n_launches;    /* kernels this context has launched (all entry points)       */
    int32_t drop_schedule; /* NTVS_SCHED_PLAIN, _WINDOW or _PIPELINE (chosen at load)      */
    int32_t lanes_per_row; /* lanes per row of the DROP kernel                           */
    int64_t n_escaped;     /* DELTA16: 32-entry chunks stored with full columns          */
    int32_t voxel_tile_x;  /* internal voxel tile of the loaded system (1 = canonical)   */
    int32_t voxel_tile_y;
} ntvs_stats;

/* Device time of the context's kernels, measured with CUDA events recorded on the
 * context's stream around every launch while profiling is on. */
typedef struct {
    double drop_block_ms;     /* DROP gather + scatter kernels (step a5)                 */
    int64_t drop_block_launches;
    double drop_apply_ms;     /* x += delta / s kernels (step a6)                         */
    int64_t drop_apply_launches;
    double tv_ms;             /* TV gradient, value and perturbation kernels              */
    int64_t tv_launches;
} ntvs_profile;

/* Library version string. */
const char* ntvs_version(void);

/* Message of the calling thread's last failed call ("" if none). */
const char* ntvs_last_error(void);

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t to queue
 * work on (e.g. a torch.cuda.Stream's cuda_stream), or NULL for a non-blocking stream the
 * context creates and owns; pass cudaStreamLegacy ((void*)0x1) to queue on the legacy
 * default stream.  *out is NULL on failure. */
int ntvs_create(ntvs_ctx** out, int device, void* cuda_stream);

/* Destroy a context (synchronizes its stream, frees its device memory).  NULL is a no-op. */
int ntvs_destroy(ntvs_ctx* ctx);

/* Load (replace) the system.  Validates it on the device (row_ptr non-decreasing from 0,
 * col in [0,V), finite val and b), computes ||a_i||^2 in FP64 from the stored values,
 * the block partition and the per-block hit counts s_j^t, and packs DELTA16 storage.
 * Resets the image to 0, the cycle counter k and ell_{k-1} to 0 and the traces.
 * Errors: NTVS_ERR_ARG (sizes, dtypes, V > 2^31-1), NTVS_ERR_CSR (validation),
 * NTVS_ERR_OOM, NTVS_ERR_CUDA.  Synchronous. */
int ntvs_load_system(ntvs_ctx* ctx, const ntvs_system* sys);

/* A system given as proton paths instead of a stored matrix: row i of A is traced from
 * history i's path every DROP sweep (Sec. I: rows are the intersection lengths of each
 * tracked proton with the voxels).  Path record i (10 floats, mm): chord start P_in (x,y,z),
 * chord end P_out (x,y,z), offsets (A_lat, B_lat, A_z, B_z); the path is
 *   P(s) = P_in + s (P_out - P_in) + (A_lat h10(s) + B_lat h11(s)) n + (A_z h10(s) + B_z h11(s)) e_z
 * for s in [0,1], h10 = s^3 - 2 s^2 + s, h11 = s^3 - s^2, n = (-u_y, u_x, 0) the in-plane unit
 * normal of the chord, cut into n_seg straight segments.  Each segment is cut at the voxel
 * planes it crosses and each piece (FP32 geometry) is credited to the voxel holding its
 * midpoint; pieces shorter than min_len are dropped.  Voxels are dx x dy x dz with the grid
 * origin at (-nx dx/2, -ny dy/2, 0). */
typedef struct {
    int32_t nx, ny, nz;
    int32_t n_blocks;            /* contiguous blocks of ceil(M/B) rows when block_ptr is NULL */
    double dx, dy, dz;           /* voxel size (mm)                                            */
    int64_t n_rows;              /* M                                                          */
    const float* paths;          /* [M][10] path records (mem_kind)                            */
    const float* b;              /* [M] WEPL (mem_kind)                                        */
    const int64_t* block_ptr;    /* NULL or [B+1] HOST array                                   */
    int32_t n_seg;               /* straight segments per path, 1..64                          */
    int32_t mem_kind;            /* NTVS_MEM_HOST (copied) | NTVS_MEM_DEVICE (borrowed)        */
    double min_len;              /* pieces shorter than this are dropped (mm), >= 0            */
} ntvs_paths;

/* Load (replace) the system as paths (FP32 arithmetic).  At load one thread per row
 * traces the path, merges the pieces of one voxel at segment joins and computes ||a_i||^2
 * (FP64) and the hit counts s_j^t; every DROP sweep traces the paths again.  Resets the
 * image and the run state like ntvs_load_system.  Errors: NTVS_ERR_ARG, NTVS_ERR_CSR
 * (non-finite path or b), NTVS_ERR_OOM, NTVS_ERR_CUDA. */
int ntvs_load_paths(ntvs_ctx* ctx, const ntvs_paths* p);

/* The same system given by the tracking data of each history (Sec. I: every proton is
 * tracked and its most likely path predicted from that data).  History i (12 floats, mm):
 * entry point P_in (x,y,z), exit point P_out (x,y,z), entry direction d_in and exit
 * direction d_out (any length; a zero vector stands for the chord
 * direction).  Its path is the cubic Hermite curve from P_in to P_out with end tangents
 * L d_in/|d_in| and L d_out/|d_out|, L = |P_out - P_in| (the paper's most likely path is not
 * defined in it; this curve stands in for it).  The curve is stored in the path-record form
 * of ntvs_load_paths: the tangents' deviations from the chord, m - (P_out - P_in), are
 * projected on the chord's in-plane normal n (A_lat, B_lat) and on z (A_z, B_z); their
 * component along the chord's in-plane direction, which only re-times the walk along the
 * curve, is dropped.  The conversion runs on the device; everything else is
 * ntvs_load_paths.  The paper has no counterpart for this format. */
typedef struct {
    int32_t nx, ny, nz;
    int32_t n_blocks;            /* contiguous blocks of ceil(M/B) rows when block_ptr is NULL */
    double dx, dy, dz;           /* voxel size (mm)                                            */
    int64_t n_rows;              /* M                                                          */
    const float* hist;           /* [M][12] P_in, P_out, d_in, d_out (mem_kind; read at load)  */
    const float* b;              /* [M] WEPL (mem_kind; device b is borrowed, host b copied)   */
    const int64_t* block_ptr;    /* NULL or [B+1] HOST array                                   */
    int32_t n_seg;               /* straight segments per path, 1..64                          */
    int32_t mem_kind;            /* NTVS_MEM_HOST | NTVS_MEM_DEVICE                            */
    double min_len;              /* pieces shorter than this are dropped (mm), >= 0            */
} ntvs_histories;

/* Load (replace) the system from history data; the context keeps the converted path
 * records (40 B per history) and, for host input, its own copy of b.  Errors as
 * ntvs_load_paths (NTVS_ERR_CSR for a non-finite history value or b). */
int ntvs_load_histories(ntvs_ctx* ctx, const ntvs_histories* h);

/* Set the NTVS parameters (Appendix C).  Validated: N >= 0, 0 < alpha < 1, beta0 >= 0,
 * eps_tv >= 0, lambda finite, max_retries >= 1 when tv_check.  Default before the first
 * call: lambda 1e-4, alpha 0.75, beta0 1, eps_tv 1e-8, N 0, no check, 64 retries, seed 0. */
int ntvs_set_params(ntvs_ctx* ctx, const ntvs_params* p);

/* Set the current image x (the initial iterate x-bar of Appendix A) from V values of
 * `dtype` (NTVS_F64 or NTVS_F32) in host or device memory. */
int ntvs_set_image(ntvs_ctx* ctx, const void* x, int dtype, int mem_kind);

/* Copy the current image into V values of `dtype` (NTVS_F64 or NTVS_F32). */
int ntvs_get_image(ntvs_ctx* ctx, void* out, int dtype, int mem_kind);

/* Run k_iters cycles of NTVS from the current state (Appendix C): per cycle
 * ell_k = rand(k, ell_{k-1}); N perturbation steps x <- x + beta0*alpha^ell v, ell++
 * (with the check: retry with ell++ until phi(z) <= phi(x), at most max_retries tries,
 * beta recomputed after every try); then x <- P_T(x); then phi(x) in FP64.
 * The call only queues work.  With the check (NTVS and OTVS rules) every decision is
 * taken on the device: ell_k is drawn there and each step's retry loop runs in one
 * cooperative kernel, so no try waits for the host; the traces, the counters of
 * ntvs_get_stats and ell_{k-1} stay on the device until one of ntvs_get_stats,
 * ntvs_get_trace, ntvs_get_state, ntvs_set_state or a run without the check needs them
 * (one synchronization then). */
int ntvs_run(ntvs_ctx* ctx, int k_iters);

/* Wait for the context's stream. */
int ntvs_sync(ntvs_ctx* ctx);

/* phi(x) of the current image, FP64 reduction on the device (synchronous). */
int ntvs_get_tv(ntvs_ctx* ctx, double* tv);

/* Counters of the run so far (synchronous). */
int ntvs_get_stats(ntvs_ctx* ctx, ntvs_stats* st);

/* Per-block residual sums of squares sum_i (b_i - <a_i,x>)^2 (FP64, x before the block's
 * update) of the last DROP sweep; out has room for `cap` >= n_blocks doubles. */
int ntvs_get_block_resid(ntvs_ctx* ctx, double* out, int cap);

/* Traces of the run so far: ell_k per cycle ([k] entries), and per perturbation step
 * the tries and whether x changed ([k*N] entries).  *n receives the number written;
 * any output pointer may be NULL. */
int ntvs_get_trace(ntvs_ctx* ctx, int64_t* ell_k, int32_t* tries, int32_t* accepted,
                   int64_t cap, int64_t* n_cycles);

/* Checkpoint state besides the image: cycle counter k and ell_{k-1}.  Restoring
 * (k, ell_prev) and the image resumes a run exactly where it stopped. */
int ntvs_get_state(ntvs_ctx* ctx, int64_t* k, int64_t* ell_prev);
int ntvs_set_state(ntvs_ctx* ctx, int64_t k, int64_t ell_prev);

/* Turn per-launch event timing on (1) or off (0); turning it on clears the totals. */
int ntvs_set_profiling(ntvs_ctx* ctx, int on);

/* Totals of the launches timed since profiling was turned on (synchronizes the stream). */
int ntvs_get_profile(ntvs_ctx* ctx, ntvs_profile* out);

/* Internal voxel order of the FP32 path, applied at the next ntvs_load_system: the FP32
 * gather copy of x, the DROP accumulator and the hit counts are stored in in-plane tiles
 * of tx x ty voxels (each tile contiguous, slices contiguous), and the stored columns are
 * rewritten into that order on the device (into a buffer of the context's own when the
 * caller's columns are device memory: they are never modified).  Rows of a proton history
 * then touch fewer distinct cache lines per slice.  For stored systems the in-slice
 * offsets are also permuted inside each aligned group of 32 (the shared-memory bank
 * spread of the slice-windowed DROP kernels; a group stays on its 128-byte line).  The
 * results are those of the canonical order up to the order of floating-point
 * accumulation; images, gradients and every other public array stay canonical.  tx, ty
 * in {1, 2, 4, 8, 16}; 1 x 1 leaves the in-plane order canonical; the default is 4 x 4.
 * It applies to ntvs_load_paths and ntvs_load_histories too (the traced voxel indices are
 * formed in the tiled order, without the in-group permutation); the FP64 path always uses
 * the canonical order.  This layout has no counterpart in the paper.
 * NTVS_ERR_ARG on other sizes. */
int ntvs_set_voxel_tile(ntvs_ctx* ctx, int tx, int ty);

/* Arithmetic of systems loaded with FP32 values, applied at the next ntvs_load_system:
 * NTVS_F32 (default) computes dot products, scatters, the TV gradient and the image
 * copies in FP32 (FP64 only for the decision-making reductions); NTVS_F64 computes every
 * step in FP64 on the FP32-stored values and b (b is widened to FP64 once at load), as the
 * FP64 path does for FP64 storage, while the matrix streams at 8 bytes per entry.  FP64
 * systems always use FP64 arithmetic and FP16/BF16 systems FP32 arithmetic (NTVS_F64
 * leaves them unchanged).  Why the option exists: NTVS with a small eps_tv amplifies
 * perturbations of the image below sqrt(eps_tv) from one cycle to the next, so FP32
 * rounding (relative 6e-8 per operation) grows to ~1e-4 relative L2 after 12 cycles at
 * eps_tv = 1e-8; the FP64 oracle itself moves as far when b is perturbed by 6e-8.  FP64
 * arithmetic keeps the result within ~1e-10 of the FP64 reference.  This choice has no
 * counterpart in the paper.  NTVS_ERR_ARG for other values. */
int ntvs_set_compute_dtype(ntvs_ctx* ctx, int dtype);

/* Test hook: replay ell_k for the next n cycles instead of drawing it (NULL clears). */

/* Failure-detection test hook.  Every device-side wait of the library (the pipelined DROP
 * kernel's mbarrier waits, the TV-check loop's grid barrier) gives up after wait_ns
 * nanoseconds (wait_ns <= 0: the default, 2 s), records an error code and lets its CTA
 * leave with no copy in flight; the next synchronizing call returns NTVS_ERR_TIMEOUT and
 * the image of that run is invalid, while the context stays usable.  flags make a wait run
 * out on purpose: NTVS_HOOK_STARVE_PIPE (the pipelined schedule's producer withholds the
 * first stage of every CTA) and NTVS_HOOK_STARVE_CHECK (the first CTA of the TV-check
 * loop withholds its first barrier arrival).  0 restores normal operation.  Nothing here
 * has a counterpart in the paper.  NTVS_ERR_ARG for unknown flags. */
#define NTVS_HOOK_STARVE_PIPE 1
#define NTVS_HOOK_STARVE_CHECK 2
int ntvs_set_fault_hook(ntvs_ctx* ctx, int64_t wait_ns, int flags);

int ntvs_set_ell_override(ntvs_ctx* ctx, const int64_t* ell_k, int64_t n);

/* ---- single steps of the hot path (same kernels as ntvs_run) ---------------------- */

/* g = grad phi_eps(x) of the current image into V values of `dtype` (NTVS_F64/F32);
 * *gnorm (may be NULL) receives ||g||_2 from the FP64 device reduction.  Synchronous. */
int ntvs_tv_gradient(ntvs_ctx* ctx, void* g_out, int dtype, int mem_kind, double* gnorm);

/* One perturbation step without the check: x <- x - beta * g/||g|| (Appendix C). */
int ntvs_perturb(ntvs_ctx* ctx, double beta);

/* One try with the check: z = x - beta g/||g||; if phi(z) <= phi(x) then x <- z.
 * *accepted receives 1 or 0; *phi_x / *phi_z (may be NULL) the FP64 values.  Synchronous. */
int ntvs_perturb_checked(ntvs_ctx* ctx, double beta, int* accepted, double* phi_x, double* phi_z);

/* One DROP block t in [0, B) on the current image (queued); its residual sum of squares
 * is readable afterwards with ntvs_get_block_resid. */
int ntvs_drop_block(ntvs_ctx* ctx, int t);

/* One full DROP sweep P_T (blocks 0..B-1 in order). */
int ntvs_drop_sweep(ntvs_ctx* ctx);

/* Forward projection: out[i] = <a_i, x> for every row i of the loaded system (the stored
 * values, or the traced paths of ntvs_load_paths / ntvs_load_histories exactly as the DROP
 * sweeps trace them), in the context's compute precision.  x: V values of x_dtype
 * (NTVS_F64 / NTVS_F32, canonical order, host or device); out: M values of out_dtype (host
 * or device, caller-owned).  The current image is not touched.  Allocates temporaries;
 * synchronous.  The rows are the paper's system (Sec. I, Sec. III-D); the entry point
 * itself (e.g. for synthetic right-hand sides b = A x) has no counterpart in the paper. */
int ntvs_forward_project(ntvs_ctx* ctx, const void* x, int x_dtype, int x_mem, void* out, int out_dtype, int out_mem);

/* ---- row-sharded DROP ---------------------------------------------------------------
 * All rows of a block see the same x (Sec. III-D, block-DROP of ref. CEHN08), so the rows
 * of every block may be split over several GPUs: each forms the sum over its rows,
 *     delta_j = lambda * sum_{i in its rows of block t} a_ij (b_i - <a_i, x>) / ||a_i||^2,
 * the deltas are summed over the GPUs, and each applies x_j += delta_j / s_j^t with the
 * GLOBAL hit count s_j^t of the block.  The paper runs on one GPU (Sec. IV); this split is
 * the library's own.  The library never reads another GPU's memory: the sums are the
 * caller's collective (e.g. NCCL). */

/* Element type of hit counts in the all-reduce callback. */
#define NTVS_I32 4

/* delta of rows [r0, r1) of block t (r0 = r1 = -1: all of the block's rows; otherwise
 * block_ptr[t] <= r0 <= r1 <= block_ptr[t+1]) on the current image, NOT applied: V values
 * of dtype (NTVS_F32 / NTVS_F64) in canonical voxel order into delta_out (caller-owned,
 * host or device).  *resid_ss (may be NULL) receives sum (b_i - <a_i, x>)^2 over those rows
 * (FP64).  A proper sub-range runs the plain schedule.  Synchronous for host output or
 * resid_ss, else queued.  Errors: NTVS_ERR_ARG, NTVS_ERR_STATE, NTVS_ERR_CUDA. */
int ntvs_drop_block_partial(ntvs_ctx* ctx, int t, int64_t r0, int64_t r1, void* delta_out, int dtype, int mem_kind,
                            double* resid_ss);

/* x_j += delta[j] / s_j^t for an externally summed delta (V values of dtype, canonical
 * order, host or device) with the context's hit counts of block t (see below). */
int ntvs_apply_delta(ntvs_ctx* ctx, int t, const void* delta, int dtype, int mem_kind);

/* The hit counts s_j^t of block t (V int32, canonical order, host or device): the counts
 * of this context's rows after ntvs_load_system; a shard replaces them by the sum over all
 * shards before applying deltas.  Counts must be >= 0. */
int ntvs_get_hit_counts(ntvs_ctx* ctx, int t, int32_t* out, int mem_kind);
int ntvs_set_hit_counts(ntvs_ctx* ctx, int t, const int32_t* counts, int mem_kind);

/* Collective of a row-sharded reconstruction: sum buf[0..n) (device memory, element type
 * dtype: NTVS_F32, NTVS_F64 or NTVS_I32) over all ranks in place, queued on cuda_stream
 * (the context's stream) so that work queued after it sees the sum; return 0 on success.
 * Every rank must make the same sequence of calls. */
typedef int (*ntvs_allreduce_fn)(void* buf, int64_t n, int dtype, void* cuda_stream, void* user);

/* Turn the context into one rank of a row-sharded reconstruction.  Call it on every rank
 * after ntvs_load_system with that rank's rows (same grid, blocks, parameters, voxel tile
 * and image on every rank).  It sums the hit counts of all blocks over the ranks through fn
 * once (every rank then holds the global counts), and from then on every DROP block of
 * ntvs_run / ntvs_drop_sweep / ntvs_drop_block sums the block's delta (the internal-order
 * accumulator, n = the padded voxel count) and its residual sum of squares through fn
 * before applying them.  The TV steps run on every rank on identical images.  fn = NULL
 * leaves sharded mode (the counts stay global until the next load).  Loading a system
 * clears the callback.  Errors: NTVS_ERR_STATE (no system, or a callback already set),
 * NTVS_ERR_CUDA (fn returned nonzero). */
int ntvs_set_allreduce(ntvs_ctx* ctx, ntvs_allreduce_fn fn, void* user);

/* ---- batched reconstructions ----------------------------------------------------------
 * Many independent NTVS reconstructions (Appendix C) advanced together on one GPU: every
 * member has its own grid, system, blocks and parameters, with or without the TV check
 * (Sec. III-E).  A cycle of all members is two kernel launches replayed from a CUDA graph:
 * a setup kernel, and one persistent kernel whose CTAs take work items (runs of voxels or
 * of DROP rows of one member's current phase) from per-member counters; the last item of
 * a phase publishes the member's next phase, so members overlap and none waits for the
 * others.  A CTA that finds no item polls for at most the hook's wait (2 s by default);
 * when that runs out the cycle stops and the next synchronizing call returns
 * NTVS_ERR_TIMEOUT (the images are then undefined: destroy the batch).  Members without
 * the check take their step sizes beta_{k,n} from the host (the ell schedule of
 * ntvs_run, copied in per cycle); checked members draw ell_k on the device and try up
 * to max_retries step sizes, four per pass.  Members take FP32 values in CSR32 storage,
 * given as a matrix (ntvs_batch_add) or traced on the device from path records
 * (ntvs_batch_add_paths); all preparation (validation, norms, hit counts) runs on the
 * device.  Arithmetic as the single-context FP32 path: FP32 rows and gathers, FP64 image,
 * reductions in a fixed order. */
typedef struct ntvs_batch ntvs_batch;

typedef struct {
    int32_t members;            /* reconstructions in the batch                          */
    int32_t lanes_per_row;      /* largest DROP lanes per row of any member (8, 16, 32)   */
    int64_t cycles;             /* cycles run                                             */
    int64_t n_launches;         /* kernels launched by ntvs_batch_run                     */
    int64_t kernels_per_cycle;  /* kernels in one cycle's graph (2)                       */
    int64_t total_rows, total_nnz, total_voxels;
    int32_t rows_per_item;      /* DROP rows per work item (tuned at finalize)           */
    int32_t window_floats;      /* shared scatter window per CTA, 0: global scatter      */
    int32_t ctas;               /* CTAs of the persistent kernel                          */
    int32_t lanes_per_row_min;  /* smallest DROP lanes per row of any member              */
    int32_t ctas_per_sm;        /* register fit of the persistent kernel (3 or 4 CTAs/SM) */
    int32_t lanes_per_row_all;  /* lanes per row of every member picked by the tuning, 0:
                                   each member's own (from its mean row length)             */
} ntvs_batch_stats;

/* Test hook of the batch (ntvs_batch_set_fault_hook): member 0 never leaves its first
 * phase, so every other CTA runs out of work and the bounded wait ends the cycle. */
#define NTVS_HOOK_STARVE_BATCH 4

int ntvs_batch_create(ntvs_batch** out, int device, void* cuda_stream);
int ntvs_batch_destroy(ntvs_batch* bt);
/* Add a member: system (val_dtype NTVS_F32, storage NTVS_CSR32, host or device arrays,
 * copied and validated on the device), parameters and initial image x0 (V values, F64 or
 * F32, host or device).  *index (may be NULL) receives the member's index.  Before
 * finalize only.  Errors: NTVS_ERR_ARG, NTVS_ERR_CSR (row_ptr, columns, non-finite
 * values), NTVS_ERR_STATE, NTVS_ERR_OOM, NTVS_ERR_CUDA. */
int ntvs_batch_add(ntvs_batch* bt, const ntvs_system* sys, const ntvs_params* p, const void* x0, int x0_dtype,
                   int x0_mem, int* index);
/* Add a member given as path records (the format of ntvs_load_paths): its rows are traced
 * once on the device (one thread per history, the path's pieces in order, consecutive
 * pieces of one voxel merged, merged pieces shorter than min_len dropped) and stored as
 * FP32 CSR32.  Errors as ntvs_batch_add (NTVS_ERR_CSR for a non-finite path value or b). */
int ntvs_batch_add_paths(ntvs_batch* bt, const ntvs_paths* paths, const ntvs_params* p, const void* x0,
                         int x0_dtype, int x0_mem, int* index);
/* Fix the persistent kernel's schedule instead of timing candidates at finalize:
 * rows_per_item > 0 DROP rows per work item (0: tuned), window_floats >= 0 floats of the
 * shared scatter window (0: global scatter only; -1: tuned).  Before finalize only. */
int ntvs_batch_set_schedule(ntvs_batch* bt, int rows_per_item, int window_floats);
/* Bounded-wait limit (wait_ns > 0; 0 restores 2 s) and test hooks (NTVS_HOOK_STARVE_BATCH)
 * of the cycles run after finalize.  Before finalize only.  The paper has no counterpart. */
int ntvs_batch_set_fault_hook(ntvs_batch* bt, int64_t wait_ns, int flags);
/* Lay out the work tables, pick the schedule (ntvs_batch_set_schedule, or by timing one
 * cycle of each candidate: rows per item {256, 512, 1024} x window {0, 8192, 12288, 16384} x
 * {3, 4} CTAs per SM, then on the best of those the rows per warp: lanes per row 32, 16
 * or 8 for every member against each member's own; images restored afterwards) and
 * capture the cycle graph; max_cycles bounds the cycles that may be run (per-member phi
 * history). */
int ntvs_batch_finalize(ntvs_batch* bt, int max_cycles);
/* Queue k_iters cycles of every member on the batch's stream. */
int ntvs_batch_run(ntvs_batch* bt, int k_iters);
/* Wait for the queued cycles; NTVS_ERR_TIMEOUT when a bounded wait ran out. */
int ntvs_batch_sync(ntvs_batch* bt);
/* Member `index`'s image (synchronous); phi after its last cycle (FP64). */
int ntvs_batch_get_image(ntvs_batch* bt, int index, void* out, int dtype, int mem_kind);
int ntvs_batch_get_tv(ntvs_batch* bt, int index, double* tv);
/* Member `index`'s counters (synchronous): out5 = {cycles, ell (ell_{k-1} of the next
 * cycle), TV steps, accepted steps, tries}. */
int ntvs_batch_get_member(ntvs_batch* bt, int index, int64_t* out5);
/* Member `index`'s stored rows (synchronous; host arrays, each may be NULL): n_rows, nnz,
 * row_ptr [M+1], col [nnz] (canonical voxel index), val [nnz]. */
int ntvs_batch_get_rows(ntvs_batch* bt, int index, int64_t* n_rows, int64_t* nnz, int64_t* row_ptr, int32_t* col,
                        float* val);
int ntvs_batch_get_stats(ntvs_batch* bt, ntvs_batch_stats* st);
/* The schedule candidates timed at finalize: *n of them (0 when the schedule was fixed);
 * the first min(*n, cap) are written as cand[4i..4i+3] = (rows per item, window floats,
 * CTAs per SM, lanes per row of every member or 0 for each member's own) and ms[i] = its
 * cycle time (ms). */
int ntvs_batch_get_tuning(ntvs_batch* bt, int32_t* cand, float* ms, int cap, int* n);

/* ---- allocation-free entry point --------------------------------------------------- */

/* phi(x) of a caller-owned image, for callers that cannot allocate device memory: code
 * that runs inside a host callback or a framework hook where allocating is not allowed,
 * under an allocator that must own every device allocation of the process, or with a
 * device-memory budget fixed in advance.  The paper has no counterpart; it computes the
 * same FP64 value as ntvs_get_tv, without a context.
 *   x       : device pointer, V = nx*ny*nz values of `dtype` (NTVS_F64 or NTVS_F32),
 *             layout [nz][ny][nx]; on the current CUDA device.
 *   tv_out  : device pointer to one double, written when the stream reaches the kernel.
 *   cuda_stream : cudaStream_t to queue on (NULL = the default stream).
 * Nothing is allocated: the reduction scratch (4096 FP64 partials and a ticket word) is a
 * static device array that every GPU loading the library holds until the process exits.
 * Limit: V <= 16,777,216 voxels (4096 CTAs x 256 threads x 16 voxels); larger images
 * return NTVS_ERR_ARG.  Every call looks up the scratch's device address in the current
 * context (cudaGetSymbolAddress, which allocates nothing); the first call on a device also
 * loads the library's device code there, so make that first call before any stream
 * capture.  All calls share the one scratch array, which keeps the last call's
 * contents: calls that overlap on the GPU (other streams, other threads) race and give
 * wrong results, so order them on one stream.  Errors: NTVS_ERR_ARG, NTVS_ERR_CUDA. */
int ntvs_tv_value_static(const void* x, int dtype, int nx, int ny, int nz, double* tv_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* NTVS_H */
