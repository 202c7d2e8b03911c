// Device building blocks: memory-ordering primitives, the bounded grid
// barrier, per-warp asynchronous staging, and the 32-row-tile SpMV used by
// every solver phase ("MV" in Section 3 / Table 1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace bcs {

constexpr unsigned kFull = 0xffffffffu;

// ---- memory ordering -------------------------------------------------------

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_gpu_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_int(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// system scope (several GPUs meeting at one barrier through peer memory)
__device__ __forceinline__ unsigned ld_acquire_sys(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_sys_add(unsigned* p, unsigned v) {
    asm volatile("red.release.sys.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_int_sys(const int* p) {
    int v;
    asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative (co-resident) launch.  A monotonic
// arrival counter: barrier k completes when the counter reaches k*gridDim.
// Arrival is a release reduction, the wait an acquire load, so every write
// made before the barrier by any CTA is visible after it.  The wait is
// bounded: past `budget` cycles (or when another CTA has already failed) the
// CTA records BCS_ERR_TIMEOUT and the call returns false; callers then leave
// the kernel, so a missing CTA can never hang the GPU.  SYS: the CTAs of
// several GPUs meet at a counter in one GPU's memory (release/acquire at
// system scope, so that their stores into each other's memory are visible
// after the barrier); `epoch` starts at the barriers already passed on that
// counter (it is not reset between solves).
template <bool SYS>
struct GridBarrierT {
    unsigned* count;
    int* err;
    unsigned nblocks;
    unsigned epoch;
    long long budget;

    __device__ bool sync(volatile int* s_flag) {
        __syncthreads();
        if (threadIdx.x == 0) {
            epoch += 1;
            const unsigned target = epoch * nblocks;
            if constexpr (SYS) red_release_sys_add(count, 1u);
            else red_release_gpu_add(count, 1u);
            int ok = 1;
            const long long t0 = clock64();
            while ((int)((SYS ? ld_acquire_sys(count) : ld_acquire_gpu(count)) - target) < 0) {
                if ((SYS ? ld_relaxed_int_sys(err) : ld_relaxed_int(err)) != 0) { ok = 0; break; }
                if (clock64() - t0 > budget) {
                    if constexpr (SYS) atomicCAS_system(err, 0, (int)BCS_ERR_TIMEOUT);
                    else atomicCAS(err, 0, (int)BCS_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
            *s_flag = ok;
        }
        __syncthreads();
        return *s_flag != 0;
    }
};
using GridBarrier = GridBarrierT<false>;

// ---- L2 eviction priority ----------------------------------------------------------
// Streams that are not read again before L2 would have dropped them anyway
// (the matrix, which is larger than L2 on the large systems, and Krylov
// vectors whose next use is an iteration away) are loaded and stored with an
// evict_first policy, so that in L2 they give way to the vectors that the
// next phase of the iteration reads again.  A policy is a hint: it changes
// no value.
__device__ __forceinline__ unsigned long long l2_first() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Solves use the hints only when the vectors that the next phase re-reads fit
// in L2 together (KParams::l2hint, decided on the host from the system size;
// the kernels are instantiated with and without them, H): hints that cannot
// keep the re-read set resident were measured to cost time, and so did a
// run-time choice inside the tile loops (a branch per load, or both code
// paths in the loop body).
__device__ __forceinline__ int ldg_first(const int32_t* p, unsigned long long pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double ldv_first(const double* p, unsigned long long pol) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ldv_first(const float* p, unsigned long long pol) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ldv_first(const uint16_t* p, unsigned long long pol) {
    unsigned short v;
    asm("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
    return __uint_as_float(((unsigned)v) << 16);
}
// plain (coherent) load and store of a Krylov vector element with the policy
__device__ __forceinline__ double ld_first(const double* p, unsigned long long pol) {
    double v;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol) : "memory");
    return v;
}
__device__ __forceinline__ float ld_first(const float* p, unsigned long long pol) {
    float v;
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol) : "memory");
    return v;
}
__device__ __forceinline__ void st_first(double* p, double v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_first(float* p, float v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
// ---- value types ---------------------------------------------------------------

__device__ __forceinline__ double ldv(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldv(const float* p) { return __ldg(p); }
// BF16 bit pattern -> float (exact: BF16 is the top half of an FP32).
__device__ __forceinline__ float ldv(const uint16_t* p) {
    return __uint_as_float(((unsigned)__ldg((const unsigned short*)p)) << 16);
}
// The hints are used with FP32 vectors only, and then only on systems whose
// re-read set fits in L2 (8 x 8.4 MB on the 2.1M-row system: the hints cut
// the DRAM traffic of an iteration by a quarter).  With FP64 vectors that
// set is larger than L2 on the large systems and the hints were measured to
// add traffic, so FP64 solves load and store without them.
template <class VT>
__host__ __device__ constexpr bool l2_hints() { return sizeof(VT) == 4; }
// Matrix loads of a tile: H (compile time) = with the evict_first policy pol.
template <bool H>
__device__ __forceinline__ int ldg_col(const int32_t* p, unsigned long long pol) {
    if constexpr (H) return ldg_first(p, pol);
    else return __ldg(p);
}
template <bool H, class VT, class MT>
__device__ __forceinline__ VT ldg_val(const MT* p, unsigned long long pol) {
    if constexpr (H) return (VT)ldv_first(p, pol);
    else return (VT)ldv(p);
}

__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// device-wide nanosecond clock (the same on every SM)
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Per-warp double-buffered staging of the 32-row chunks of up to kMaxStage
// vectors.  Every lane copies its own row of each vector with cp.async
// (global -> shared without going through registers, coalesced across the
// warp like a load) and commits one group per stage; a lane waits only for
// its own copies (cp.async.wait_group) and reads back only its own row, so no
// cross-lane synchronisation and no spin is involved.  The source vectors
// must be padded to whole 32-row tiles (the solver's arena is).
constexpr int kMaxStage = 12;

template <class VT>
__device__ __forceinline__ void cp_async_elem(VT* dst, const VT* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(sizeof(VT))
                 : "memory");
}
template <class VT>
__device__ __forceinline__ void cp_async_elem_first(VT* dst, const VT* src, unsigned long long pol) {
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], %2, %3;" ::"r"(smem_addr(dst)), "l"(src),
                 "n"(sizeof(VT)), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <class VT>
struct WarpStager {
    VT* buf;                   // [2][kMaxStage][32] in shared memory
    unsigned pending;          // bit s: stage s has a committed group not yet waited for

    // FIRST: bit k set = vector k is not read again before L2 drops it (evict_first)
    template <unsigned FIRST = 0u, bool H = false, int K>
    __device__ __forceinline__ void issue(const VT* const (&v)[K], int64_t tile, int stage,
                                          unsigned long long pol = 0ull) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            VT* const d = buf + (stage * kMaxStage + k) * 32 + lane;
            const VT* const src = v[k] + tile * 32 + lane;
            if (H && ((FIRST >> k) & 1u)) cp_async_elem_first(d, src, pol);
            else cp_async_elem(d, src);
        }
        cp_async_commit();
        pending |= 1u << stage;
    }
    // wait for `stage` (the older of the two in flight when `other` is pending)
    __device__ __forceinline__ const VT* wait(int stage) {
        if ((pending >> (stage ^ 1)) & 1u) cp_async_wait<1>(); else cp_async_wait<0>();
        pending &= ~(1u << stage);
        return buf + stage * kMaxStage * 32;
    }
    // every copy in flight has landed (before the stages are abandoned or reused out of order)
    __device__ __forceinline__ void settle() {
        cp_async_wait<0>();
        pending = 0u;
    }
};

// ---- SpMV on a tile of 32 consecutive rows (lane k -> row row0+k) -----------------

constexpr int kSpmvBatch = 8;  // entries per lane whose loads are in flight together

// CSR with T lanes per row.  T == 1: each lane sums its row sequentially in
// storage order with fma (the same order as a plain CSR loop).  T > 1: the
// T lanes of a group take strided entries of one row, then combine with a
// butterfly; 32/T rows per pass, results transposed back through shared
// memory so that lane k holds row row0+k.  Rows >= n yield 0.
template <class VT, class MT, int T, bool H>
__device__ __forceinline__ VT csr_tile(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                       const MT* __restrict__ val, const VT* x, int64_t row0, int64_t n,
                                       VT* s_buf, unsigned long long pol) {
    const int lane = threadIdx.x & 31;
    const int64_t row = row0 + lane;
    int rp0 = 0, rp1 = 0;
    if (row < n) {
        rp0 = ldg_col<H>(rowptr + row, pol);
        rp1 = ldg_col<H>(rowptr + row + 1, pol);
    }
    if constexpr (T == 1) {
        // Batches of kSpmvBatch entries: all column and value loads of the batch are
        // issued, then all gathers, then the fmas in storage order -- two memory
        // rounds per batch instead of two per entry, same rounding as a plain loop.
        VT acc = VT(0);
        for (int k0 = rp0; k0 < rp1; k0 += kSpmvBatch) {
            int c[kSpmvBatch];
            VT v[kSpmvBatch], xv[kSpmvBatch];
#pragma unroll
            for (int j = 0; j < kSpmvBatch; ++j) {
                const bool in = k0 + j < rp1;
                c[j] = in ? ldg_col<H>(col + k0 + j, pol) : 0;
                v[j] = in ? ldg_val<H, VT>(val + k0 + j, pol) : VT(0);
            }
#pragma unroll
            for (int j = 0; j < kSpmvBatch; ++j) xv[j] = (k0 + j < rp1) ? x[c[j]] : VT(0);
#pragma unroll
            for (int j = 0; j < kSpmvBatch; ++j)
                if (k0 + j < rp1) acc = vfma(v[j], xv[j], acc);
        }
        return acc;
    } else {
        constexpr int G = 32 / T;
        const int sub = lane % T, grp = lane / T;
#pragma unroll 1
        for (int pass = 0; pass < T; ++pass) {
            const int r = pass * G + grp;
            const int b = __shfl_sync(kFull, rp0, r);
            const int e = __shfl_sync(kFull, rp1, r);
            VT acc = VT(0);
#pragma unroll 2
            for (int k = b + sub; k < e; k += T) acc = vfma(ldg_val<H, VT>(val + k, pol), x[ldg_col<H>(col + k, pol)], acc);
#pragma unroll
            for (int off = T / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
            if (sub == 0) s_buf[r] = acc;
        }
        __syncwarp();
        const VT v = s_buf[lane];
        __syncwarp();
        return v;
    }
}

// SELL-C-sigma with C = 32: tile == slice, lane == row of the slice.  The
// slice is column-major, so each step reads 32 consecutive values and column
// indices (fully coalesced); each lane sums its row in storage order with fma.
// Padding (value 0, a valid column) leaves the sum unchanged.
template <class VT, class MT, bool H>
__device__ __forceinline__ VT sell_tile(const int64_t* __restrict__ slice_ptr, const int32_t* __restrict__ scol,
                                        const MT* __restrict__ sval, const VT* x, int64_t slice,
                                        unsigned long long pol) {
    const int lane = threadIdx.x & 31;
    const int64_t b = __ldg(slice_ptr + slice), e = __ldg(slice_ptr + slice + 1);
    VT acc = VT(0);
    for (int64_t k0 = b + lane; k0 < e; k0 += 32 * kSpmvBatch) {  // batched as in csr_tile
        int c[kSpmvBatch];
        VT v[kSpmvBatch], xv[kSpmvBatch];
#pragma unroll
        for (int j = 0; j < kSpmvBatch; ++j) {
            const bool in = k0 + 32 * j < e;
            c[j] = in ? ldg_col<H>(scol + k0 + 32 * j, pol) : 0;
            v[j] = in ? ldg_val<H, VT>(sval + k0 + 32 * j, pol) : VT(0);
        }
#pragma unroll
        for (int j = 0; j < kSpmvBatch; ++j) xv[j] = (k0 + 32 * j < e) ? x[c[j]] : VT(0);
#pragma unroll
        for (int j = 0; j < kSpmvBatch; ++j)
            if (k0 + 32 * j < e) acc = vfma(v[j], xv[j], acc);
    }
    return acc;
}

// CSR tile with adaptive lanes per row (T == 0): a row of at most kLongRow
// entries is summed by its own lane in storage order (as csr_tile<.., 1>);
// each longer row is summed by the whole warp (lane l takes entries l, l+32,
// ... in order, then a butterfly), so a tile with a few long rows no longer
// waits for them one entry at a time.  The long rows' sums are therefore in a
// different order than a plain sequential loop (deterministic).
constexpr int kLongRow = 32;
template <class VT, class MT, bool H>
__device__ __forceinline__ VT csr_tile_adaptive(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                const MT* __restrict__ val, const VT* x, int64_t row0, int64_t n,
                                                unsigned long long pol) {
    const int lane = threadIdx.x & 31;
    const int64_t row = row0 + lane;
    int rp0 = 0, rp1 = 0;
    if (row < n) {
        rp0 = ldg_col<H>(rowptr + row, pol);
        rp1 = ldg_col<H>(rowptr + row + 1, pol);
    }
    const bool lng = rp1 - rp0 > kLongRow;
    unsigned lmask = __ballot_sync(kFull, lng);
    const int send = lng ? rp0 : rp1;
    VT acc = VT(0);
    for (int k0 = rp0; k0 < send; k0 += kSpmvBatch) {
        int c[kSpmvBatch];
        VT v[kSpmvBatch], xv[kSpmvBatch];
#pragma unroll
        for (int j = 0; j < kSpmvBatch; ++j) {
            const bool in = k0 + j < send;
            c[j] = in ? ldg_col<H>(col + k0 + j, pol) : 0;
            v[j] = in ? ldg_val<H, VT>(val + k0 + j, pol) : VT(0);
        }
#pragma unroll
        for (int j = 0; j < kSpmvBatch; ++j) xv[j] = (k0 + j < send) ? x[c[j]] : VT(0);
#pragma unroll
        for (int j = 0; j < kSpmvBatch; ++j)
            if (k0 + j < send) acc = vfma(v[j], xv[j], acc);
    }
    while (lmask) {
        const int src = __ffs(lmask) - 1;
        lmask &= lmask - 1u;
        const int b = __shfl_sync(kFull, rp0, src), e = __shfl_sync(kFull, rp1, src);
        VT part = VT(0);
        for (int k0 = b + lane; k0 < e; k0 += 32 * 4) {
            int c[4];
            VT v[4], xv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bool in = k0 + 32 * j < e;
                c[j] = in ? ldg_col<H>(col + k0 + 32 * j, pol) : 0;
                v[j] = in ? ldg_val<H, VT>(val + k0 + 32 * j, pol) : VT(0);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) xv[j] = (k0 + 32 * j < e) ? x[c[j]] : VT(0);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (k0 + 32 * j < e) part = vfma(v[j], xv[j], part);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(kFull, part, off);
        if (lane == src) acc = part;
    }
    return acc;
}

// CSR tile, one lane per row, with the lane's row range [rp0, rp1) already
// loaded (rows >= n: an empty range): the same entries, order and fmas as
// csr_tile<VT, MT, 1>.
template <class VT, class MT, bool H>
__device__ __forceinline__ VT csr_tile_rp(int rp0, int rp1, const int32_t* __restrict__ col,
                                          const MT* __restrict__ val, const VT* x, unsigned long long pol) {
    VT acc = VT(0);
    for (int k0 = rp0; k0 < rp1; k0 += kSpmvBatch) {
        int c[kSpmvBatch];
        VT v[kSpmvBatch], xv[kSpmvBatch];
#pragma unroll
        for (int j = 0; j < kSpmvBatch; ++j) {
            const bool in = k0 + j < rp1;
            c[j] = in ? ldg_col<H>(col + k0 + j, pol) : 0;
            v[j] = in ? ldg_val<H, VT>(val + k0 + j, pol) : VT(0);
        }
#pragma unroll
        for (int j = 0; j < kSpmvBatch; ++j) xv[j] = (k0 + j < rp1) ? x[c[j]] : VT(0);
#pragma unroll
        for (int j = 0; j < kSpmvBatch; ++j)
            if (k0 + j < rp1) acc = vfma(v[j], xv[j], acc);
    }
    return acc;
}
// H: matrix loads with the evict_first policy (FP32/BF16 vectors only)
template <class VT, class MT, int LAYOUT, int T, bool H = false>
__device__ __forceinline__ VT tile_spmv(const KParams& P, const MT* val, const VT* x, int64_t tile, VT* s_buf) {
    constexpr bool kH = H && l2_hints<VT>();
    const unsigned long long pol = kH ? l2_first() : 0ull;
    if constexpr (LAYOUT == LAY_SELL) return sell_tile<VT, MT, kH>(P.slice_ptr, P.col, val, x, tile, pol);
    else if constexpr (T == 0) return csr_tile_adaptive<VT, MT, kH>(P.rowptr, P.col, val, x, tile * 32, P.n, pol);
    else return csr_tile<VT, MT, T, kH>(P.rowptr, P.col, val, x, tile * 32, P.n, s_buf, pol);
}

}  // namespace bcs
