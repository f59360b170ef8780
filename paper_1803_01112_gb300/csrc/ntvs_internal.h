// Internal launch interface between the host runtime (ntvs_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <type_traits>

namespace ntvs {

// compute / storage element types (same numbering as the public NTVS_F64 ...)
enum Dt { F64 = 0, F32 = 1, F16 = 2, BF16 = 3 };

inline size_t dt_size(int dt) { return dt == F64 ? 8 : dt == F32 ? 4 : 2; }

// Internal voxel order of the FP32 gather copy, delta, hit counts and matrix columns:
// in-plane tiles of tx x ty voxels, each tile contiguous, tiles row-major over a grid padded
// to multiples of the tile, slices contiguous (slice_p voxels each).  With sw set, the
// in-slice offset p of that order is stored at p ^ ((p >> 5) & 31): a bijection inside
// each aligned group of 32 offsets (slice_p is then a multiple of 32), which is the bank
// spread of the DROP kernels' slice windows, so that their window slot is the voxel's
// offset in its slice.  tx = ty = 1 without sw is the canonical order (iz*ny + iy)*nx + ix.
// Public images and the FP64 master stay canonical.  tx, ty are powers of two (ltx, lty
// their logarithms); V and vint stay below 2^31.
struct VoxMap {
    int nx, ny, nz;
    int nxp, nyp;      // padded to multiples of tx, ty
    int tx, ty;
    int ltx, lty;
    int sw;            // 1: offsets swizzled inside each slice
    int64_t slice_p;   // nxp * nyp, rounded up to a multiple of 32 with sw
    int64_t vint;      // nz * slice_p
};

// tx, ty powers of two
inline VoxMap make_voxmap(int nx, int ny, int nz, int tx, int ty, bool sw = false) {
    VoxMap m;
    m.nx = nx; m.ny = ny; m.nz = nz;
    m.tx = tx; m.ty = ty;
    m.ltx = 0;
    while ((1 << m.ltx) < tx) ++m.ltx;
    m.lty = 0;
    while ((1 << m.lty) < ty) ++m.lty;
    m.nxp = (nx + tx - 1) / tx * tx;
    m.nyp = (ny + ty - 1) / ty * ty;
    m.sw = sw ? 1 : 0;
    m.slice_p = (int64_t)m.nxp * m.nyp;
    if (sw) m.slice_p = (m.slice_p + 31) / 32 * 32;
    m.vint = m.slice_p * nz;
    return m;
}

// true when the internal order is not the canonical one (columns are rewritten at load)
inline bool voxmap_reorders(const VoxMap& m) { return m.tx != 1 || m.ty != 1 || m.sw; }

// internal index of canonical voxel j on the host (the device has vox_internal)
inline int64_t vox_internal_host(const VoxMap& m, int64_t j) {
    if (!voxmap_reorders(m)) return j;
    const int64_t ix = j % m.nx, t = j / m.nx, iy = t % m.ny, iz = t / m.ny;
    const int64_t ntx = m.nxp / m.tx;
    int64_t p = ((iy / m.ty) * ntx + ix / m.tx) * (int64_t)(m.tx * m.ty) + (iy % m.ty) * m.tx + ix % m.tx;
    if (m.sw) p ^= (p >> 5) & 31;
    return iz * m.slice_p + p;
}

// FP32 copies of the FP64 master image, written together with it: x32 in the internal
// voxel order (the DROP gathers), and on the FP32 path xh = fl32(x), xl = fl32(x - xh) in
// canonical order, from which the TV stencil forms neighbour differences as
// (xh_a - xh_b) + (xl_a - xl_b) in FP32 (the FP64 difference rounded to FP32 for
// neighbours within a factor of two, as good as rounding it otherwise) with no FP64
// arithmetic.  Null pointers are skipped.
struct ImgCopies {
    float* x32;
    float* xh;
    float* xl;
    VoxMap m;
};

// Grid used by every deterministic reduction: a fixed CTA count so the order of the
// final sum over CTA partials never changes.
constexpr int kRedThreads = 256;
int red_grid(int64_t n, int sm_count);

// ------------------------------------------------------------------ load-time prep
// flags |= 1 if row_ptr decreases, 2 if row_ptr[0] != 0
cudaError_t k_validate_rows(const int64_t* row_ptr, int64_t M, int* flags, cudaStream_t s);
// fused pass over the rows [r0, r1) of one block: validation of columns, values and b
// (flags 4 / 8 / 16), inv_norm2 of the rows and the block's hit counts cnt; with colsum
// (nullable) also colsum[j] += |a_ij|, rb[0] = max(rb[0], max_i |b_i| / ||a_i||^2) and
// rb[1] = max(rb[1], max |a_ij|).  col and val hold the entries from e0 on: entry p is
// col[p - e0] (0 for whole arrays, the block's first entry for a staging slot).
cudaError_t k_prep_block(const int64_t* row_ptr, const int32_t* col, const void* val, int64_t e0, int vdt,
                         const void* b, int64_t r0, int64_t r1, int64_t nvox, void* inv_norm2, int cdt, int32_t* cnt,
                         int* flags, float* colsum, float* rb, cudaStream_t s);
// *out = max(*out, max_j v[j]) for n non-negative floats
cudaError_t k_colmax(const float* v, int64_t n, float* out, cudaStream_t s);
// col_out[p] = internal index of voxel col_in[p]; flags |= 4 for a column outside [0, V)
// (written as 0).  col_in == col_out is allowed.
cudaError_t k_remap_cols(const int32_t* col_in, int32_t* col_out, int64_t nnz, VoxMap m, int* flags, cudaStream_t s);
// x32[internal(j)] = (float)x[j] for the canonical voxels j < V
cudaError_t k_x32_from_x64(const double* x, ImgCopies c, cudaStream_t s);
// inv_s[j] = cnt[j] ? 1/cnt[j] : 0
cudaError_t k_inv_counts(const int32_t* cnt, void* inv_s, int cdt, int64_t n, cudaStream_t s);

// DELTA16 index storage: every row is cut into chunks of 32 entries from its first entry;
// chunk k of row i (entries p0 + 32k ..) has slot (p0 >> 5) + i + k (no two chunks share a
// slot, since a row of n entries has at most n/32 + 1 chunks) and stores base cbase[slot] =
// its smallest column, every entry the 16-bit offset off[p] = col[p] - base.  A chunk whose
// columns span more than 65535 is escaped: cbase[slot] = -1 - e and its columns are
// exc[32 e + (p - p0 - 32k)].  rowesc[i] bit 0: row i has an escaped chunk (only those rows
// pay for the check; the others decode every column with one add); bit 1: row i is narrow
// (its columns span at most 65535: every chunk base is the row's smallest column, so the
// windowed kernel loads the base once per row).  With 16-bit values the offset and the
// value's bits share one word (offset in the low half), read with one 4-byte load.
struct Delta16 {
    const uint16_t* off;      // [nnz] (FP32/FP64 values)
    const int32_t* cbase;     // [(nnz >> 5) + M + 1]
    const int32_t* exc;       // [escaped chunks][32]
    const uint8_t* rowesc;    // [M]
    const uint32_t* word;     // [nnz] 16-bit values: offset | value bits << 16 (off and val unused)
};
// DELTA16 storage with 16-bit (FP16/BF16) values keeps each entry as one 32-bit word
template <typename V, bool D16>
__host__ __device__ constexpr bool delta16_words() { return D16 && sizeof(V) == 2; }
cudaError_t k_pack_words(const uint16_t* off, const uint16_t* val, int64_t n, uint32_t* word, cudaStream_t s);
// slots of the chunk bases for nnz entries in M rows
inline int64_t delta16_slots(int64_t nnz, int64_t M) { return (nnz >> 5) + M + 1; }
// escaped chunks: *n_esc += their number (zeroed by the caller)
cudaError_t k_delta16_count(const int64_t* row_ptr, const int32_t* col, int64_t M, unsigned long long* n_esc,
                            cudaStream_t s);
// writes off, cbase, exc and rowesc (escape slots taken from *slot, zeroed by the caller)
cudaError_t k_delta16_fill(const int64_t* row_ptr, const int32_t* col, int64_t M, uint16_t* off, int32_t* cbase,
                           int32_t* exc, uint8_t* rowesc, unsigned long long* slot, cudaStream_t s);

// ------------------------------------------------------------------ TV
// Scratch of the deterministic reductions: partials[2*grid] doubles and a ticket word
// that the last CTA resets to 0.
struct RedScratch {
    double* partials;
    unsigned* ticket;
    int grid;
};

// The image x is always the FP64 master copy; g and the stencil arithmetic use cdt.
// g = grad phi_eps(x); *gnorm2 = ||g||^2 (FP64); if phi != nullptr also *phi = phi_0(x).
// On the FP32 path without phi the stencil reads xh/xl (when not null) instead of x.
cudaError_t k_tv_grad(int cdt, const double* x, const float* xh, const float* xl, void* g, int nx, int ny, int nz,
                      double eps, RedScratch r, double* gnorm2, double* phi, cudaStream_t s);
// *phi = phi_0(z), z = x - sc*g with sc = beta/sqrt(*gnorm2) (z = x when g == nullptr or
// gnorm2 == 0).  If phi_ref != nullptr, *accept = (*phi <= *phi_ref).
cudaError_t k_tv_value(int cdt, const double* x, const void* g, const double* gnorm2, double beta, int nx, int ny,
                       int nz, RedScratch r, double* phi, const double* phi_ref, int* accept, cudaStream_t s);
// x <- x - sc*g (sc as in k_tv_value) and its FP32 copies; skipped when accept != nullptr
// and *accept == 0.
cudaError_t k_tv_apply(int cdt, double* x, ImgCopies c, const void* g, const double* gnorm2, double beta,
                       const int* accept, int64_t V, cudaStream_t s);

// ------------------------------------------------------------------ DROP
// A run of consecutive rows [r0, r1) whose entries lie mostly in z-slice `home`.
struct DropSegment {
    int64_t r0, r1;
    int32_t home, pad;
};

// CSR32 storage with FP32 values is packed at load: entry p is the pair {column, bits of
// the value} (int2, 8 bytes), so a lane reads its entry with one load.  The DROP,
// projection and pipelined kernels take the pair array through their column pointer and
// leave the value pointer unused: a kernel on FP32 values without DELTA16 indices
// (packed_entries) reads pairs.
template <typename V, bool D16>
__host__ __device__ constexpr bool packed_entries() { return !D16 && std::is_same<V, float>::value; }
cudaError_t k_pack_entries(const int32_t* col, const float* val, int64_t n, int32_t* ent, cudaStream_t s);

struct DropArgs {
    const int64_t* row_ptr;
    const int32_t* col;    // int32 columns, or (CSR32 with FP32 values) the packed pairs
    const void* val;       // storage type vdt; unused with packed pairs
    const void* b;         // compute type
    const void* inv_norm2; // compute type
    int64_t r0, r1;
    const void* x;         // gather image: FP64 master (F64 path) or its FP32 copy (F32 path)
    void* delta;           // compute type, accumulates lambda * sum_i a_ij r_i
    double lambda;
    double* resid_ss;      // += sum_i (b_i - <a_i,x>)^2
    int vdt, cdt;
    int lanes_per_row;     // 4, 8, 16 or 32
    int grid;
    bool vector4;          // col/val 16-byte (8-byte for 2-byte values) aligned: 4-entry vector loads
    bool use_d16;          // DELTA16 index storage (d16 below) instead of col
    Delta16 d16;
    // windowed schedule (segs != nullptr): grid CTAs of 1024 threads, CTA c takes segments
    // [seg_begin[c], seg_begin[c+1]); shared window of one z-slice (slice = nx*ny voxels)
    const DropSegment* segs;
    const int32_t* seg_begin;
    int64_t slice;
    // FP32 windowed schedule: the window accumulates in int32 fixed point with quantum
    // Q = |lambda| * bound * lmax / 2^30, where lmax = max_j sum_{i in block} |a_ij| and
    // bound = *wbound (a bound on |b_i - <a_i,x>| / ||a_i||^2); rows above the bound
    // scatter with global FP32 reductions instead.  *wobs receives the block's observed
    // max of that ratio (atomic max of float bits).  All three point at block t's slot.
    const float* wlmax;
    const float* wbound;
    float* wobs;
    const float* wamax;   // max |a_ij| of the block: rows whose terms could reach 2^22 Q go global
    int64_t max_row;      // longest row of the block (register steps of the windowed kernel)
};
// dynamic shared memory of the windowed DROP kernel for a slice of `slice` voxels
int64_t k_window_smem_bytes(int64_t slice, int csz, bool d16);
cudaError_t k_drop_block(const DropArgs& a, cudaStream_t s);

// Register steps of the row body the windowed kernel runs for a block whose longest row
// has max_row entries (a warp per row, FP32 compute on FP32 or BF16 values): as many 32-entry
// steps as that row needs, 8..11, else 12 (longer rows finish in a tail loop).  Rows of at
// most kShortBody steps take the 8-step body, and in blocks deeper than kMidBody rows of at
// most kMidBody steps take a kMidBody-step body (CSR32 rows and narrow DELTA16 rows).  0: the kernel's fixed
// depth applies.
constexpr int kShortBody = 8;
constexpr int kMidBody = 10;
inline int window_register_steps(int64_t max_row, int cdt, int vdt, int lanes_per_row) {
    if (cdt != F32 || (vdt != F32 && vdt != BF16) || lanes_per_row != 32) return 0;
    const int64_t need = (max_row + 31) / 32;
    return need <= 8 ? 8 : need <= 11 ? (int)need : 12;
}
// Work of rows [cs[q], cs[q+1]) for each chunk q in quarters of an issued register step:
// per row 4 (its reductions and bookkeeping) + 4 per live step of the body it runs
// (kShortBody when it fits, else mid when it fits and mid > 0, else ch[q]) + 1 per step of
// that body past the row's end (issued predicated off: no loads, gathers or scatters) + 8
// per step past ch[q] (the tail loop reads those entries twice).  Charging empty steps a
// quarter instead of a full step measured 0.2302 -> 0.2281 ms per 500k-row block.
cudaError_t k_chunk_cost(const int64_t* row_ptr, const int64_t* cs, const int8_t* ch, int mid, int64_t nchunks,
                         int64_t* cost, int grid, cudaStream_t s);
cudaError_t k_drop_block_d16(const DropArgs& a, cudaStream_t s);   // the same on DELTA16 storage
// out[i] = <a_i, x> for the M rows (x: compute type, in the order of the stored columns;
// out: compute type); a.row_ptr, col / d16, val, vdt, cdt, use_d16 and grid are used
cudaError_t k_project(const DropArgs& a, int64_t M, const void* x, void* out, cudaStream_t s);
// *out = max(*out, longest row of rows [r0, r1)); *out zeroed by the caller
cudaError_t k_row_maxlen(const int64_t* row_ptr, int64_t r0, int64_t r1, unsigned long long* out, int grid,
                         cudaStream_t s);
// home[i] = median z-slice of the first, middle and last entries of row i (-1: empty row);
// entry p's column is col[stride * p] (2 for the packed pairs)
cudaError_t k_row_home(const int64_t* row_ptr, const int32_t* col, int stride, int64_t M, int64_t slice, int32_t* home,
                       int grid, cudaStream_t s);
// chunk q = rows [chunk_start[q], chunk_start[q+1]) (at most 64 rows): out[q] = lower median
// of the defined home slices (-1 if none); *changes += rows whose defined home differs from
// the previous row's defined home (*changes must be zeroed by the caller)
cudaError_t k_chunk_home(const int32_t* home, const int64_t* chunk_start, int64_t nchunks, int32_t* out,
                         unsigned long long* changes, int grid, cudaStream_t s);
// x_j += delta_p * inv_s_p on the FP64 master (p the internal index of j) and its FP32
// copies; delta_p = 0.  With wbound (block t's slot, nullable): *wbound = 2 * *wobs when
// the block observed a ratio (the next sweep's bound), *wobs = 0.
cudaError_t k_drop_apply(int cdt, double* x, ImgCopies c, void* delta, const void* inv_s, int64_t V, int grid,
                         float* wbound, float* wobs, cudaStream_t s);

// TMA-fed pipeline (drop_pipe_kernel): a stage is a run of at most kStageRows whole rows
// of one home slice whose entries [e0, e0 + nent) fit one ring slot (e0 and nent aligned
// to 16 bytes of both col and val); off[k] = row_ptr[r0 + k] - e0.  nent == 0 marks a
// single row too long for a slot, read from global memory.
constexpr int kStageRows = 15;
struct DropStage {
    int64_t e0;
    int64_t r0;
    int32_t nent;
    int16_t nrows;
    int16_t home;
    uint16_t off[kStageRows + 1];
    int64_t pad;
};
struct DropPipeArgs {
    const int64_t* row_ptr;
    const int32_t* col;   // int32 columns, or the packed pairs (FP32 values)
    const void* val;      // unused with packed pairs
    const void* b;
    const void* inv_norm2;
    const DropStage* stages;
    const int32_t* stage_begin;   // [grid + 1] for this block
    int64_t slice;
    const void* x;
    void* delta;
    double lambda;
    double* resid_ss;
    int* err;                     // set (nonzero) when a bounded wait runs out
    uint64_t wait_ns;             // bound of each wait
    int starve;                   // test hook: the producer withholds every CTA's first stage
    int vdt, cdt;
    int grid;
    bool use_d16;                 // DELTA16 index storage (d16) instead of col
    Delta16 d16;
};
cudaError_t k_drop_pipe(const DropPipeArgs& a, cudaStream_t s);
// entries per ring slot and dynamic shared memory, for ring_bytes bytes per entry: the
// index plus the value (int32 columns or DELTA16 offsets with separate values), or the
// single 8-byte pair or 4-byte DELTA16 word
int pipe_stage_entries(int ring_bytes);
size_t pipe_smem_bytes(int cdt, int ring_bytes, int64_t slice);

// ------------------------------------------------------------------ on-the-fly rows
struct OtfArgs {
    const float* paths;   // [M][10]
    const float* b;       // [M]
    int64_t M;
    int nx, ny, nz;
    double dx, dy, dz;
    int n_seg;
    float min_len;
    int grid;
    VoxMap vm;            // order of the traced voxel indices (x32, delta, hit counts)
};
cudaError_t k_otf_validate(const OtfArgs& a, int* flags, cudaStream_t s);
// history data [M][12] (P_in, P_out, d_in, d_out) -> path records [M][10]; flags |= 32 on a
// non-finite value
cudaError_t k_hist_to_paths(const float* hist, int64_t M, float* rec, int* flags, int grid, cudaStream_t s);
// inv_norm2 of rows [r0, r1) and the block's hit counts cnt (+= 1 per distinct voxel)
cudaError_t k_otf_prep(const OtfArgs& a, int64_t r0, int64_t r1, float* inv_norm2, int32_t* cnt, cudaStream_t s);
cudaError_t k_otf_drop(const OtfArgs& a, int64_t r0, int64_t r1, const float* inv_norm2, const float* x, float* delta,
                       double lambda, double* resid_ss, cudaStream_t s);
// out[i] = <a_i, x> of every traced row (x in the internal voxel order)
cudaError_t k_otf_project(const OtfArgs& a, const float* x, float* out, cudaStream_t s);
// stored rows from paths: entries per row, then (voxel in the order of a.vm, length) from row_ptr
cudaError_t k_otf_count_rows(const OtfArgs& a, int32_t* nnz_row, cudaStream_t s);
cudaError_t k_otf_fill_rows(const OtfArgs& a, const int64_t* row_ptr, int32_t* col, float* val, cudaStream_t s);

// ------------------------------------------------------------------ row-sharded DROP
// out[j] = delta[internal(j)] in type odt (F32/F64), then delta = 0 (canonical j < V)
cudaError_t k_delta_out(int cdt, void* delta, VoxMap m, void* out, int odt, cudaStream_t s);
// x_j += d[j] * inv_s[internal(j)], d canonical of type ddt (F32/F64), and the FP32 copies
cudaError_t k_apply_ext(int cdt, double* x, ImgCopies c, const void* d, int ddt, const void* inv_s, cudaStream_t s);
// cnt[p] = round(1 / inv_s[p]) (0 where inv_s = 0), n slots of one order
cudaError_t k_counts_from_inv(int cdt, const void* inv_s, int32_t* cnt, int64_t n, cudaStream_t s);
// canonical counts of a block from its internal-order inverse counts, and back
cudaError_t k_counts_out(int cdt, const void* inv_s, VoxMap m, int32_t* cnt, cudaStream_t s);
cudaError_t k_counts_in(int cdt, const int32_t* cnt, VoxMap m, void* inv_s, cudaStream_t s);

// ------------------------------------------------------------------ TV check on the device
// Error codes written to the device error word by bounded waits (the host reports them as
// NTVS_ERR_TIMEOUT): 1-7 the pipelined DROP kernel, 8 the TV-check loop's grid barrier.
constexpr int kErrCheckBarrier = 8;

// Device-resident state of the checked variant: the current ell (ell_{k-1} between
// cycles) and the arrival counter of the retry loop's grid barrier.
struct CheckState {
    int64_t ell;
    unsigned bar;
    int pad;
};
// ell_k of cycle k into st->ell and *ell_slot: the override when given, else ell_{k-1}
// under the OTVS rule, else rand(k, ell_{k-1}) of stream `seed`.
cudaError_t k_check_cycle_begin(CheckState* st, int rule, uint64_t seed, int64_t k, bool has_override,
                                int64_t override_ell, int64_t* ell_slot, cudaStream_t s);
struct CheckLoopArgs {
    int cdt;
    double* x;                 // FP64 master image, updated on accept
    ImgCopies copies;          // its FP32 copies (null members skipped)
    const void* g;             // gradient (compute type)
    const double* gnorm2;      // ||g||^2
    const double* phi_x;       // phi(x) of the same gradient pass
    CheckState* st;
    const double* beta_tab;    // beta0 * alpha^ell for ell < tab_len (host-computed)
    int tab_len;
    double beta0, alpha;       // beyond the table: beta0 * pow(alpha, ell) on the device
    int max_retries;
    double* partials;          // >= 2 * grid doubles
    int grid;                  // <= check_loop_max_grid (co-resident)
    int* err;
    uint64_t wait_ns;          // bound of each barrier wait
    int starve;                // test hook: CTA 0 withholds its first barrier arrival
    int32_t* tries_out;        // this step's tries and accept flag
    int32_t* acc_out;
    int nx, ny, nz;
};
cudaError_t k_tv_check_loop(const CheckLoopArgs& a, cudaStream_t s);
// largest co-resident grid of the retry-loop kernel (0 if the query fails)
int check_loop_max_grid(int cdt, int sms);

// ------------------------------------------------------------------ misc
// sets the calling thread's ntvs_last_error() text
void set_last_error(const std::string& msg);

// convert between the image's compute type and F64/F32 buffers (device to device)
cudaError_t k_convert(const void* src, int sdt, void* dst, int ddt, int64_t n, cudaStream_t s);

}  // namespace ntvs
