// Block-DROP with a TMA-fed pipeline (P_T of arXiv 1803.01112 Appendix C; DROP of ref.
// CEHN08, Sec. III-D): the same update as drop_block_window_kernel,
//     r_i = lambda (b_i - <a_i, x>) / ||a_i||^2,   delta_j += r_i a_ij,
// with the matrix stream decoupled from the dependent gather -> dot -> scatter chain.
//
// One CTA per SM.  Warp 0 is the producer: one thread walks the CTA's stage list
// (planned at load time: runs of whole rows of one home z-slice, at most kStageRows rows
// and S entries, start aligned to 16 bytes) and copies each stage's columns and values
// (for FP32 values: its packed {column, value} pairs, one copy)
// into a ring of kStages shared-memory slots with cp.async.bulk, completing on the
// slot's "full" mbarrier.  Warps 1..31 are consumers: they walk the same stages in order,
// each taking every 31st row, compute the row's dot product from shared memory (x
// gathered from L1/L2), and scatter r_i a_ij into a shared-memory window of the home
// slice (XOR-swizzled slots) or, outside the slice, into delta with global reductions.
// A consumer releases a slot by arriving on its "empty" mbarrier.  When the home slice
// changes the consumers meet on a third mbarrier and flush the window.
//
// Every wait is bounded by a %globaltimer deadline (a runtime budget, 2 s by default): on
// expiry the thread records an error code (read by the host as NTVS_ERR_TIMEOUT) and
// leaves, and the producer waits (again bounded) for each of its own copies in flight
// before it exits.  A test hook makes the producer withhold every CTA's first stage, so
// that the waits on it run out.
#include "common.cuh"

namespace ntvs {

namespace {

constexpr int kStages = 4;                      // ring slots
constexpr int kDescBatch = 32;                  // stage descriptors fetched per bulk copy
constexpr int kThreads = 1024;
constexpr int kConsumers = kThreads / 32 - 1;   // 31 consumer warps

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait (wait_ns) for the phase with the given parity; false (and *err set) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code, uint64_t wait_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() - t0 > wait_ns) {
            atomicExch(err, code);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// window slot of slice offset j: the FP32 path's internal voxel order carries the bank
// swizzle inside each slice already; the FP64 path (canonical order) XORs the low 5 bits
// with the next 5 here
template <typename T>
__device__ __forceinline__ int win_slot(int j) {
    if constexpr (sizeof(T) == 4) return j;
    else return j ^ ((j >> 5) & 31);
}

template <typename T>
__device__ __forceinline__ void scatter_w(T* win, int W, int64_t w0, T* delta, int32_t c, T v) {
    const int64_t rel = (int64_t)c - w0;
    if ((uint64_t)rel < (uint64_t)W) atomicAdd(win + win_slot<T>((int)rel), v);
    else atomicAdd(delta + c, v);
}

// entry q: int32 column + value, or a packed {column, value bits} pair (FP32 values)
template <typename T, typename V, typename IdxT>
__device__ __forceinline__ void entry_at(const IdxT* cs, const V* vs, int q, int32_t& c, T& a) {
    if constexpr (std::is_same<IdxT, int2>::value) {
        const int2 e = cs[q];
        c = e.x;
        a = (T)__int_as_float(e.y);
    } else {
        c = cs[q];
        a = (T)to_compute(vs[q]);
    }
}

// one row of a stage: entries [o0, o1) of the stage buffers (or of global memory)
template <typename T, typename V, typename IdxT>
__device__ __forceinline__ void pipe_row(const IdxT* cs, const V* vs, int o0, int o1, int64_t i, const T* b,
                                         const T* inv_norm2, const T* x, T* win, int W, int64_t w0, T* delta, T lambda,
                                         double& ss) {
    const int lane = threadIdx.x & 31;
    const T bi = __ldg(b + i), ni = __ldg(inv_norm2 + i);
    T acc = (T)0;
#pragma unroll 4
    for (int q = o0 + lane; q < o1; q += 32) {
        int32_t c;
        T a;
        entry_at<T, V, IdxT>(cs, vs, q, c, a);
        acc += a * __ldg(x + c);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const T res = bi - acc;
    const T r = lambda * res * ni;
    if (lane == 0) ss += (double)res * (double)res;
#pragma unroll 4
    for (int q = o0 + lane; q < o1; q += 32) {
        int32_t c;
        T a;
        entry_at<T, V, IdxT>(cs, vs, q, c, a);
        scatter_w(win, W, w0, delta, c, r * a);
    }
}

// the same on DELTA16 storage: cs holds the row's 16-bit column offsets, cs[o0] being the
// row's first entry, system entry g0 + o0; entry q's column adds the base of its chunk,
// slot (p0 >> 5) + i + (q - o0) / 32, or comes from the escape table
__device__ __forceinline__ int32_t d16_col_of(const Delta16& d, const int32_t* cbr, int rel, int o) {
    const int32_t base = __ldg(cbr + (rel >> 5));
    return base >= 0 ? base + o : __ldg(d.exc + ((int64_t)(-1 - base) << 5) + (rel & 31));
}

// entry q's offset and value: a 16-bit offset with a separate value, or a DELTA16 word
template <typename T, typename V, typename IdxT>
__device__ __forceinline__ void offset_at(const IdxT* cs, const V* vs, int q, int& o, T& a) {
    if constexpr (std::is_same<IdxT, uint32_t>::value) {
        const uint32_t e = cs[q];
        o = (int)(e & 0xffffu);
        a = (T)word_value<V>(e);
    } else {
        o = cs[q];
        a = (T)to_compute(vs[q]);
    }
}

template <typename T, typename V, typename IdxT>
__device__ __forceinline__ void pipe_row_d16(const IdxT* cs, const V* vs, int o0, int o1, int64_t g0, int64_t i,
                                             const Delta16& d16, const T* b, const T* inv_norm2, const T* x, T* win,
                                             int W, int64_t w0, T* delta, T lambda, double& ss) {
    const int lane = threadIdx.x & 31;
    const T bi = __ldg(b + i), ni = __ldg(inv_norm2 + i);
    const int32_t* cbr = d16.cbase + ((g0 + o0) >> 5) + i;
    T acc = (T)0;
#pragma unroll 4
    for (int q = o0 + lane; q < o1; q += 32) {
        int o;
        T a;
        offset_at<T, V, IdxT>(cs, vs, q, o, a);
        acc += a * __ldg(x + d16_col_of(d16, cbr, q - o0, o));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const T res = bi - acc;
    const T r = lambda * res * ni;
    if (lane == 0) ss += (double)res * (double)res;
#pragma unroll 4
    for (int q = o0 + lane; q < o1; q += 32) {
        int o;
        T a;
        offset_at<T, V, IdxT>(cs, vs, q, o, a);
        scatter_w(win, W, w0, delta, d16_col_of(d16, cbr, q - o0, o), r * a);
    }
}

template <typename T>
__device__ __forceinline__ void flush_w(T* win, int Wp, T* delta, int64_t w0, int tid, int nthreads) {
    for (int jj = tid; jj < Wp; jj += nthreads) {
        const T v = win[jj];
        if (v != (T)0) {
            atomicAdd(delta + w0 + win_slot<T>(jj), v);   // the slot map is its own inverse
            win[jj] = (T)0;
        }
    }
}

template <typename T, typename V, typename IdxT>
__global__ void __launch_bounds__(kThreads, 1)
drop_pipe_kernel(const int64_t* __restrict__ row_ptr, const IdxT* __restrict__ col, const V* __restrict__ val,
                 const T* __restrict__ b, const T* __restrict__ inv_norm2, const DropStage* __restrict__ stages,
                 const int32_t* __restrict__ stage_begin, int64_t slice, int S, const T* __restrict__ x,
                 T* __restrict__ delta, T lambda, double* resid_ss, int* err, uint64_t wait_ns, int starve,
                 Delta16 d16) {
    constexpr bool kW = std::is_same<IdxT, uint32_t>::value;   // DELTA16 words
    constexpr bool kD16 = sizeof(IdxT) == 2 || kW;
    constexpr bool kPk = std::is_same<IdxT, int2>::value;      // packed pairs
    constexpr bool kNoVal = kPk || kW;                         // values inside the index ring
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int W = (int)slice;
    const int Wp = (W + 31) & ~31;
    // layout: window | ring of columns (or pairs) | ring of values | 2 x kDescBatch descriptors | mbarriers
    T* win = reinterpret_cast<T*>(smem_raw);
    IdxT* ring_c = reinterpret_cast<IdxT*>(smem_raw + (size_t)Wp * sizeof(T));
    V* ring_v = reinterpret_cast<V*>(reinterpret_cast<unsigned char*>(ring_c) + (size_t)kStages * S * sizeof(IdxT));
    DropStage* desc = reinterpret_cast<DropStage*>(reinterpret_cast<unsigned char*>(ring_v) +
                                                   (kNoVal ? (size_t)0 : (size_t)kStages * S * sizeof(V)));
    uint64_t* bars = reinterpret_cast<uint64_t*>(desc + 2 * kDescBatch);
    uint64_t* full = bars;
    uint64_t* empty = bars + kStages;
    uint64_t* cbar = bars + 2 * kStages;
    uint64_t* dbar = bars + 2 * kStages + 1;   // [2]: descriptor batches

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int j = 0; j < kStages; ++j) {
            mbar_init(full + j, 1);
            mbar_init(empty + j, kConsumers);
        }
        mbar_init(cbar, kConsumers);
        mbar_init(dbar, 1);
        mbar_init(dbar + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int j = tid; j < Wp; j += kThreads) win[j] = (T)0;
    __syncthreads();

    const int s0 = stage_begin[blockIdx.x], s1 = stage_begin[blockIdx.x + 1];
    const int n = s1 - s0;
    const int nb = (n + kDescBatch - 1) / kDescBatch;

    if (warp == 0) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            auto load_batch = [&](int m) {
                const int cnt = min(kDescBatch, n - m * kDescBatch);
                const uint32_t bytes = (uint32_t)cnt * (uint32_t)sizeof(DropStage);
                mbar_arrive_expect_tx(dbar + (m & 1), bytes);
                bulk_g2s(desc + (m & 1) * kDescBatch, stages + s0 + (size_t)m * kDescBatch, bytes, dbar + (m & 1));
            };
            int issued_b = 0, waited_b = 0;   // descriptor batches issued / waited for
            if (nb > 0) { load_batch(0); issued_b = 1; }
            if (nb > 1) { load_batch(1); issued_b = 2; }
            int k = 0;
            bool ok = true;
            for (; k < n; ++k) {
                const int m = k / kDescBatch;
                if (k % kDescBatch == 0) {
                    ok = mbar_wait(dbar + (m & 1), (m >> 1) & 1, err, 6, wait_ns);
                    if (!ok) break;
                    waited_b = m + 1;
                }
                const int slot = k % kStages;
                if (k >= kStages && !(ok = mbar_wait(empty + slot, ((k / kStages) - 1) & 1, err, 1, wait_ns))) break;
                // every consumer is past stage 32m - 1: batch m - 1's buffer may take batch m + 1
                if (k % kDescBatch == kStages - 1 && m >= 1 && m + 1 < nb) { load_batch(m + 1); issued_b = m + 2; }
                const DropStage& st = desc[(m & 1) * kDescBatch + (k % kDescBatch)];
                if (k == 0 && starve) {
                    // test hook: stage 0 is withheld, so every wait on it runs out
                } else if (st.nent > 0) {
                    const uint32_t bc = (uint32_t)st.nent * (uint32_t)sizeof(IdxT);
                    const uint32_t bv = kNoVal ? 0u : (uint32_t)st.nent * (uint32_t)sizeof(V);
                    mbar_arrive_expect_tx(full + slot, bc + bv);
                    bulk_g2s(ring_c + (size_t)slot * S, col + st.e0, bc, full + slot);
                    if (!kNoVal) bulk_g2s(ring_v + (size_t)slot * S, val + st.e0, bv, full + slot);
                } else {
                    mbar_arrive(full + slot);   // rows read straight from global memory
                }
            }
            // copies possibly still landing: the last issued stages and unconsumed batches; every
            // one is waited for (bounded) even after another wait ran out, so no copy is in
            // flight when the CTA exits (a withheld stage has none)
            for (int j = (k > kStages ? k - kStages : 0); j < k; ++j)
                if (!(j == 0 && starve)) mbar_wait(full + (j % kStages), (j / kStages) & 1, err, 2, wait_ns);
            for (int m = waited_b; m < issued_b; ++m) mbar_wait(dbar + (m & 1), (m >> 1) & 1, err, 7, wait_ns);
            (void)ok;
        }
        return;
    }

    // -------------------------------------------------------------------- consumers
    const int cw = warp - 1;
    const int ctid = tid - 32;
    const int cthreads = kThreads - 32;
    double ss = 0.0;
    int64_t next = cw;      // index (in this CTA's row sequence) of this warp's next row
    int64_t base = 0;       // row-sequence index of the current stage's first row
    int cur = -1;
    uint32_t cphase = 0;
    bool ok = true;
    for (int k = 0; k < n && ok; ++k) {
        const int slot = k % kStages;
        ok = mbar_wait(full + slot, (k / kStages) & 1, err, 4, wait_ns);
        if (!ok) break;
        const DropStage& st = desc[((k / kDescBatch) & 1) * kDescBatch + (k % kDescBatch)];
        const int home = st.home, nrows = st.nrows, nent = st.nent;
        const int64_t r0 = st.r0;
        if (home != cur) {
            if (cur >= 0) {   // flush the window of the previous slice (all consumers)
                __syncwarp();
                if (lane == 0) mbar_arrive(cbar);
                ok = mbar_wait(cbar, cphase & 1, err, 3, wait_ns);
                cphase++;
                if (!ok) break;
                flush_w(win, Wp, delta, (int64_t)cur * slice, ctid, cthreads);
                __syncwarp();
                if (lane == 0) mbar_arrive(cbar);
                ok = mbar_wait(cbar, cphase & 1, err, 3, wait_ns);
                cphase++;
                if (!ok) break;
            }
            cur = home;
        }
        const int64_t w0 = (int64_t)cur * slice;
        while (next < base + nrows) {
            const int j = (int)(next - base);
            const int64_t i = r0 + j;
            if constexpr (kD16) {
                if (nent > 0) {
                    pipe_row_d16<T, V, IdxT>(ring_c + (size_t)slot * S, kNoVal ? nullptr : ring_v + (size_t)slot * S,
                                             st.off[j], st.off[j + 1], st.e0, i, d16, b, inv_norm2, x, win, W, w0,
                                             delta, lambda, ss);
                } else {
                    const int64_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
                    pipe_row_d16<T, V, IdxT>(col + p0, kNoVal ? nullptr : val + p0, 0, (int)(p1 - p0), p0, i, d16, b,
                                             inv_norm2, x, win, W, w0, delta, lambda, ss);
                }
            } else {
                if (nent > 0) {
                    pipe_row<T, V, IdxT>(ring_c + (size_t)slot * S, kPk ? nullptr : ring_v + (size_t)slot * S,
                                         st.off[j], st.off[j + 1], i, b, inv_norm2, x, win, W, w0, delta, lambda, ss);
                } else {
                    const int64_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
                    pipe_row<T, V, IdxT>(col + p0, kPk ? nullptr : val + p0, 0, (int)(p1 - p0), i, b, inv_norm2, x,
                                         win, W, w0, delta, lambda, ss);
                }
            }
            next += kConsumers;
        }
        base += nrows;
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + slot);
    }
    if (ok && cur >= 0) {
        __syncwarp();
        if (lane == 0) mbar_arrive(cbar);
        if (mbar_wait(cbar, cphase & 1, err, 5, wait_ns)) flush_w(win, Wp, delta, (int64_t)cur * slice, ctid, cthreads);
    }
    if (lane == 0 && ss != 0.0) atomicAdd(resid_ss, ss);
}

}  // namespace

int pipe_stage_entries(int ring_bytes) {
    // ring of kStages slots, 64 KB in total, slot length a multiple of 8 entries
    const int per = ring_bytes;
    return ((65536 / (kStages * per)) / 8) * 8;
}

size_t pipe_smem_bytes(int cdt, int ring_bytes, int64_t slice) {
    const size_t Wp = (size_t)((slice + 31) & ~31LL);
    const size_t S = (size_t)pipe_stage_entries(ring_bytes);
    return Wp * dt_size(cdt) + kStages * S * (size_t)ring_bytes + 2 * kDescBatch * sizeof(DropStage) +
           (2 * kStages + 3) * sizeof(uint64_t);
}

template <typename T, typename V, typename IdxT>
static cudaError_t launch_pipe_idx(const DropPipeArgs& a, const IdxT* col, cudaStream_t s) {
    auto kern = drop_pipe_kernel<T, V, IdxT>;
    // bytes per entry in the rings: the pairs and the words carry their values
    constexpr int ring_bytes = (std::is_same<IdxT, int2>::value || std::is_same<IdxT, uint32_t>::value)
                                   ? (int)sizeof(IdxT) : (int)(sizeof(IdxT) + sizeof(V));
    const size_t smem = pipe_smem_bytes(a.cdt, ring_bytes, a.slice);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.grid, kThreads, smem, s>>>(a.row_ptr, col, (const V*)a.val, (const T*)a.b, (const T*)a.inv_norm2,
                                         a.stages, a.stage_begin, a.slice, pipe_stage_entries(ring_bytes),
                                         (const T*)a.x, (T*)a.delta, (T)a.lambda, a.resid_ss, a.err, a.wait_ns,
                                         a.starve, a.d16);
    return cudaGetLastError();
}

template <typename T, typename V>
static cudaError_t launch_pipe(const DropPipeArgs& a, cudaStream_t s) {
    if (a.use_d16) {
        if constexpr (delta16_words<V, true>()) return launch_pipe_idx<T, V, uint32_t>(a, a.d16.word, s);
        else return launch_pipe_idx<T, V, uint16_t>(a, a.d16.off, s);
    }
    if constexpr (packed_entries<V, false>())
        return launch_pipe_idx<T, V, int2>(a, reinterpret_cast<const int2*>(a.col), s);
    else
        return launch_pipe_idx<T, V, int32_t>(a, a.col, s);
}

cudaError_t k_drop_pipe(const DropPipeArgs& a, cudaStream_t s) {
    if (a.cdt == F64) {   // FP64 arithmetic on FP64 or FP32 storage
        if (a.vdt == F64) return launch_pipe<double, double>(a, s);
        if (a.vdt == F32) return launch_pipe<double, float>(a, s);
        return cudaErrorInvalidValue;
    }
    switch (a.vdt) {
        case F32: return launch_pipe<float, float>(a, s);
        case F16: return launch_pipe<float, __half>(a, s);
        case BF16: return launch_pipe<float, __nv_bfloat16>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntvs
