// The persistent solver kernel: one cooperative launch runs a whole solve
// (set-up, every iteration of Algorithm 3, 4 or 5, the FP64 true-residual
// checks and, in the refinement modes, the outer FP64 refinement loop).
//
// Mapping: warps own 32-row tiles (statically tile t -> warp t mod #warps;
// for matrices with heavy-tailed rows the warps claim tiles from a counter),
// lane k of a tile owns row 32t+k in every phase, so all vector updates are
// row-local and coalesced.  Inner products accumulate per lane (exact
// integer windows in FP64, FP64 sums in the refinement modes), are summed
// exactly per warp and per CTA into one record per CTA; after a grid barrier
// every CTA sums all records in the same exact way, so the scalars are
// bitwise identical in every CTA and no CTA ever has to broadcast them.
//
// p-BiCGSafe (Alg. 4) per iteration i, two grid barriers:
//   phase A  warps 1-9 pull the records of iteration i towards L1 and sum
//            them while the other warps compute A s_i for their first tile
//            (the overlap of the inner-product reduction with MV, Section 3);
//            warp 0 forms beta, alpha, zeta, eta and the stop test; then
//            for every tile: A s_i and the fused recurrences for p, o, u, q, w, t, z,
//            y_{i+1}, x_{i+1}, r_{i+1}; A s_i is stored for phase C;
//            partials of (y,y) (y,r) (r*,r) (r*,t) (r,r).          -- barrier
//   phase C  A w_i; q = As + beta l, g' = zeta As + eta g, s' = s - alpha q
//            (the same expressions as in phase A), l = q - Aw,
//            g_{i+1} = g' - alpha Aw, s_{i+1} = s' - g_{i+1};
//            partials of (s,s) (s,y) (s,r) (r*,s).                -- barrier
// ssBiCGSafe2 (Alg. 3), three barriers: A: s = A r + partials of s; B: the
// reduction (not overlapped) -> scalars, p, o, u; C: w = A u, t, z, y, x, r.
// p-BiCGSafe-rr (Alg. 5): on i mod m = 0, 0 < i < M the iteration instead
// runs p,o,u | w = A u, t, z, y, x | r = b - A x, l = A t, g = A y | s = A r.
//
// Every multiply-add the paper writes as "a + b*c" is one fma with the
// operands in the order of the CPU reference formulation, so that with one
// lane per CSR row (or SELL) the only rounding differences from a plain
// sequential FP64 implementation are in the inner products.
#pragma once
#include <math.h>

#include <type_traits>

#include "device.cuh"
#include "xacc.cuh"

namespace bcs {

// ---- exact inner-product partials ------------------------------------------------------
// Per-CTA records: NSLOT slots x (anchor, w2, w1, w0) as four 64-bit words.
constexpr int kRec = 4;


// Shared scratch of the block-level reductions: one exact accumulator per
// slot and warp.
template <int NW>
struct XStage {
    static_assert(NW >= 1 && NW <= 32, "one warp combines a slot");
    XAcc w[10][NW];
};

template <class ACC>
__device__ __forceinline__ void wa_init10(ACC (&a)[10]) {
#pragma unroll
    for (int k = 0; k < 10; ++k) wa_init(a[k]);
}

__device__ __forceinline__ void store_rec(unsigned long long* rec, int k, const XAcc& t) {
    rec[k * kRec + 0] = (unsigned long long)(long long)t.e;
    rec[k * kRec + 1] = t.w2;
    rec[k * kRec + 2] = t.w1;
    rec[k * kRec + 3] = t.w0;
}
__device__ __forceinline__ XAcc load_rec(const unsigned long long* r) {
    XAcc t;
    t.e = (int)(long long)r[0];
    t.w2 = r[1];
    t.w1 = r[2];
    t.w0 = r[3];
    return t;
}

// Sum the CTA's warp accumulators of the slots in MASK exactly and store them
// as the CTA's record; slots in ZMASK are recorded as empty (zero).  Warp
// k mod NW combines slot k, so the slots are combined in parallel.
template <unsigned MASK, unsigned ZMASK = 0u, int NW, class ACC>
__device__ __forceinline__ void flush_partials(ACC (&a)[10], XStage<NW>& st, unsigned long long* rec) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        if ((MASK >> k) & 1u) {
            const XAcc t = wa_warp_total(a[k]);
            if (lane == 0) st.w[k][warp] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        if (warp == k % NW) {
            if ((MASK >> k) & 1u) {
                XAcc t;
                if (lane < NW) t = st.w[k][lane]; else xa_init(t);
                t = xa_warp_aligned_sum(t);
                if (lane == 0) store_rec(rec, k, t);
            } else if ((ZMASK >> k) & 1u) {
                if (lane == 0) {
                    XAcc z;
                    xa_init(z);
                    store_rec(rec, k, z);
                }
            }
        }
    }
    __syncthreads();
}

// Sum every CTA's record exactly (all CTAs obtain the same values) and round
// each slot once: out[k] = correctly rounded slot k, for the first NS slots.
// One warp per slot: its lanes take the records c = lane, lane + 32, ...; the
// slot's common anchor is the largest record anchor, every record is shifted
// to it and the lanes add plain 192-bit integers (records are below 2^136,
// so 2^17 of them cannot overflow), then a warp sum and one rounding.
// reduce_issue pulls the slot's records into L1 ahead of reduce_finish, so
// that the caller can overlap that memory round trip with other work.
// OFF: slot k is taken by warp k + OFF (warps below OFF are left free for
// other work); OFF + NS <= NW or OFF = 0.
template <int NS, int NW, int OFF = 0>
__device__ __forceinline__ void reduce_issue(const unsigned long long* base, int nblk) {
    static_assert(NS >= 1 && NS <= 10, "slots");
    static_assert(OFF == 0 || OFF + NS <= NW, "offset slots must fit");
    const int lane = threadIdx.x & 31, warp = (threadIdx.x >> 5) - OFF;
    if (warp < 0) return;
    for (int k = warp; k < NS; k += NW)
        for (int c = lane; c < nblk; c += 32)
            asm volatile("prefetch.global.L1 [%0];" ::"l"(base + k * kRec + (size_t)c * NSLOT * kRec));
}

template <int NS, int NW, int OFF = 0>
__device__ __forceinline__ void reduce_finish(const unsigned long long* base, int nblk, XStage<NW>& st, double* out) {
    const int lane = threadIdx.x & 31, warp = (threadIdx.x >> 5) - OFF;
    (void)st;
#pragma unroll 1
    for (int k = (warp < 0 ? NS : warp); k < NS; k += NW) {
        const unsigned long long* rk = base + k * kRec;
        int E = kXaEmpty;
        for (int c = lane; c < nblk; c += 32) {
            const int e = (int)(long long)rk[(size_t)c * NSLOT * kRec];
            E = e > E ? e : E;
        }
        E = warp_max_int(E);
        double res;
        if (E == kXaNaN) {
            res = __longlong_as_double(0x7FF8000000000000ll);
        } else if (E == kXaEmpty) {
            res = 0.0;
        } else {
            XAcc a;
            a.e = E;
            a.w2 = a.w1 = a.w0 = 0ull;
            for (int c = lane; c < nblk; c += 32) {
                XAcc t = load_rec(rk + (size_t)c * NSLOT * kRec);
                if (t.e == kXaEmpty) continue;
                xa_sar192(t, E - t.e);
                xa_add192(a, t.w2, t.w1, t.w0);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long b0 = __shfl_xor_sync(0xffffffffu, a.w0, off);
                const unsigned long long b1 = __shfl_xor_sync(0xffffffffu, a.w1, off);
                const unsigned long long b2 = __shfl_xor_sync(0xffffffffu, a.w2, off);
                xa_add192(a, b2, b1, b0);
            }
            xa_norm(a);
            res = xa_round(a);
        }
        if (lane == 0) out[k] = res;
    }
    __syncthreads();
}

template <int NS, int NW>
__device__ __forceinline__ void reduce_partials(const unsigned long long* base, int nblk, XStage<NW>& st, double* out) {
    reduce_issue<NS, NW>(base, nblk);
    reduce_finish<NS, NW>(base, nblk, st, out);
}

// A set of CTAs that solve one system together: the whole cooperative grid
// (one large system) or one thread-block cluster (batched solves).
// rank/size: the CTA's place among all CTAs that write inner-product records
// and meet at the barriers; trank/tsize (when >= 0): its place among the CTAs
// that share the tiles of one row block (a rank of a partitioned solve).
template <bool SYS>
struct GridGroupT {
    GridBarrierT<SYS> gb;
    int rank, size;
    int nsync = 0;   // grid barriers passed (reported with the result)
    int trank = -1, tsize = -1;
    __device__ int tile_rank() const { return trank >= 0 ? trank : rank; }
    __device__ int tile_size() const { return tsize >= 0 ? tsize : size; }
    __device__ bool sync(volatile int* flag) {
        ++nsync;
        return gb.sync(flag);
    }
};
using GridGroup = GridGroupT<false>;
struct ClusterGroup {
    int rank, size;
    int nsync = 0;
    __device__ int tile_rank() const { return rank; }
    __device__ int tile_size() const { return size; }
    // barrier.cluster with release/acquire semantics: every write of the
    // cluster's threads before the barrier is visible after it.  All CTAs of
    // a cluster are co-scheduled, so the wait always ends.
    __device__ bool sync(volatile int*) {
        ++nsync;
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        return true;
    }
};

// DIST: a rank of a partitioned solve (bcs_dist.h): CSR rows of its own block,
// columns in its offset space, and every value that another rank's next
// matrix-vector product gathers pushed into that rank's halo as it is written.
// H: the L2 evict_first policy on the matrix and the single-use vector
// streams (FP32/BF16 vectors; instantiated for CSR with one lane per row).
// BJ: block-Jacobi right preconditioning (bcs.h, BCS_PRECOND_BLOCK_JACOBI):
// the method runs on A M^-1; every vector that a product gathers is also
// written as M^-1 v by the pass that writes it (blocks of P.bs rows lie inside
// the 32-row tiles, so the warp that holds a tile's values forms them), and
// the products gather those copies.  The solved system's iterate y is x64;
// the caller turns x = M^-1 y after the launch (CSR, one lane per row, static
// tile order; all three kinds).
// HI: FP64 inner-product terms placed 12 bits higher in their windows (wa_acc
// shift 14 instead of 2), for solves whose warps add at most 64 products per lane.
template <class VT, class MT, int LAYOUT, int T, int NW, bool DYN, class Group, bool DIST = false, bool H = false,
          bool BJ = false, bool HI = false>
__device__ __forceinline__ void solve_body(const KParams& P, Group& grp) {
    __shared__ XStage<NW> s_x;
    __shared__ double s_sum[10];
    __shared__ double s_sc[4];
    __shared__ double s_q[5];   // quotients and sqrt of the scalar recurrence
    __shared__ int s_ctl[2];
    __shared__ int s_flag;
    __shared__ VT s_buf[NW][32];
    __shared__ double s_buf64[NW][32];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gwarp = (int64_t)grp.tile_rank() * NW + warp;
    const int64_t nwarps = (int64_t)grp.tile_size() * NW;
    const int64_t n = P.n, ntiles = P.ntiles;
    const int nblk = grp.size;
    const int rank = grp.rank;
    // the CTA that writes the result block and the history: CTA 0, or in a
    // partitioned solve the first CTA of every rank (each rank's process keeps
    // its own copy; ranks of one launch write the same values)
    const bool writer = DIST ? grp.tile_rank() == 0 : rank == 0;
    const int kind = P.kind;
    const bool mixed = P.mixed != 0;
    // with enough warps the grid reduction leaves warp 0 (the scalar recurrence)
    // and warp 10 (the square root) free
    constexpr int kRedOff = NW >= 11 ? 1 : 0;
    constexpr int kSqrtWarp = NW >= 11 ? 10 : 1;

    VT* const R = (VT*)P.vec[V_R];
    VT* const RS = (VT*)P.vec[V_RS];
    VT* const Y = (VT*)P.vec[V_Y];
    VT* const Tv = (VT*)P.vec[V_T];
    VT* const Pv = (VT*)P.vec[V_P];
    VT* const U = (VT*)P.vec[V_U];
    VT* const Z = (VT*)P.vec[V_Z];
    VT* const W = (VT*)P.vec[V_W];
    VT* const L = (VT*)P.vec[V_L];
    VT* const G = (VT*)P.vec[V_G];
    VT* const O = (VT*)P.vec[V_O];
    VT* const BinW = (VT*)P.vec[V_BIN];
    VT* sCur = (VT*)P.vec[V_S];
    VT* sNxt = (VT*)P.vec[V_S2];
    int sCurId = V_S, sNxtId = V_S2;   // their vector ids (peers swap in step)
    // The inner system A x_in = b_in: (x64, b64) in FP64 mode, (d, r_outer) in refinement mode.
    VT* const X = mixed ? (VT*)P.vec[V_D] : (VT*)(void*)P.x64;
    const VT* const Bin = mixed ? (const VT*)BinW : (const VT*)(const void*)P.b64;
    const int xId = mixed ? (int)V_D : (int)NVEC;
    const MT* const val = (const MT*)P.val;
    // left shift of the FP64 products in the exact inner-product windows (wa_acc)
    constexpr int was = HI ? 14 : 2;
    // row index inside a tile loop: 32-bit with FP32 vectors (fewer address
    // instructions per tile, measured faster); 64-bit with FP64 vectors, where
    // the 32-bit form was measured slower.  n < 2^31 (checked at upload).
    using RowT = typename std::conditional<sizeof(VT) == 4, int, int64_t>::type;
    VT* const sbuf = s_buf[warp];
    double* const sbuf64 = s_buf64[warp];

    auto spmv = [&](const VT* xv, int64_t tile) -> VT {
        return tile_spmv<VT, MT, LAYOUT, T, H>(P, val, xv, tile, sbuf);
    };
    auto spmv64 = [&](const double* xv, int64_t tile) -> double {
        return tile_spmv<double, double, LAYOUT, T>(P, P.val64, xv, tile, sbuf64);
    };
    // block-Jacobi: the M^-1 copies of r, s (two, alternating like s), w and u,
    // and for the replacement step's products those of t, y and the iterate
    VT* const RH = BJ ? (VT*)P.hat[0] : nullptr;
    VT* SHc = BJ ? (VT*)P.hat[1] : nullptr;
    VT* SHn = BJ ? (VT*)P.hat[2] : nullptr;
    VT* const WH = BJ ? (VT*)P.hat[3] : nullptr;
    VT* const UH = BJ ? (VT*)P.hat[4] : nullptr;
    VT* const TH = BJ ? (VT*)P.hat[5] : nullptr;
    VT* const YH = BJ ? (VT*)P.hat[6] : nullptr;
    VT* const XH = BJ ? (VT*)P.hat[7] : nullptr;
    const VT* const BJE = (const VT*)P.bj;
    // (M^-1 v) on this lane's row, M^-1 stored [rows][bs] in block columns: the
    // block's values come from the lanes of the same block by shuffles and are
    // summed with fma in column order from zero.  Every lane of the warp calls
    // it; rows >= n pass v = 0 (their stored entries are zero as well).
    auto bj_apply = [&](const auto* E, auto v, RowT row) {
        using ET = decltype(v);
        const int bs = P.bs;
        const int base = lane & ~(bs - 1);
        const ET* e = E + (size_t)row * bs;
        ET acc = ET(0);
        for (int j = 0; j < bs; ++j) acc = vfma(e[j], __shfl_sync(0xffffffffu, v, base + j), acc);
        return acc;
    };
    // partitioned solve: a value that another rank's next matrix-vector
    // product gathers is stored straight into that rank's halo (vector id v,
    // NVEC for the FP64 x); the barrier before the product makes it visible
    auto push = [&](int v, int64_t tile, RowT row, auto val) {
        if constexpr (DIST) {
            using ET = decltype(val);
            if (__ldg(P.tile_send + tile)) {
                const int a = __ldg(P.send_ptr + row), b = __ldg(P.send_ptr + row + 1);
                for (int k = a; k < b; ++k) {
                    const int2 d = P.send_dst[k];
                    ((ET*)P.peer_vec[d.x * (NVEC + 1) + v])[d.y] = val;
                }
            }
        } else {
            (void)v; (void)tile; (void)row; (void)val;
        }
    };
    unsigned long long* const precs = (unsigned long long*)P.partials;
    auto rbase = [&](int buf) -> unsigned long long* { return precs + (size_t)buf * nblk * NSLOT * kRec; };
    auto myrec = [&](int buf) -> unsigned long long* { return rbase(buf) + (size_t)rank * NSLOT * kRec; };

    // Per-warp asynchronous staging of the row-local vector chunks of the warp's
    // next tiles (double-buffered in dynamic shared memory; see WarpStager).
    extern __shared__ __align__(128) unsigned char s_dyn[];
    WarpStager<VT> stg;
    stg.buf = (VT*)(s_dyn + (size_t)warp * 2 * kMaxStage * 32 * sizeof(VT));
    stg.pending = 0u;

    // CSR with one lane per row, FP32 vectors: the row range of the lane's row
    // in the warp's next tile is loaded one tile ahead, so the SpMV of a tile
    // starts with its column and value loads (in FP64 mode the two extra
    // registers cost more than the latency they hide)
    constexpr bool kRp = (LAYOUT == LAY_CSR && T == 1 && sizeof(VT) == 4);
    // L2 policy of the matrix and of the single-use vector streams (see l2_first)
    constexpr bool kH = H && l2_hints<VT>();
    const unsigned long long polv = kH ? l2_first() : 0ull;
    auto rp_load = [&](int64_t t, int& a, int& b) {
        a = 0; b = 0;
        const int64_t r = t * 32 + lane;
        if (t < ntiles && r < n) {
            a = __ldg(P.rowptr + r);
            b = __ldg(P.rowptr + r + 1);
        }
    };
    auto spmv_rp = [&](const VT* xv, int64_t tile, int a, int b) -> VT {
        if constexpr (kRp) return csr_tile_rp<VT, MT, kH>(a, b, P.col, val, xv, polv);
        else return spmv(xv, tile);
    };
    // Tile order of an iteration phase.  Static: tile t belongs to warp t mod
    // nwarps.  Dynamic: the warps claim tiles from a per-phase counter (one
    // atomic per tile, issued a tile ahead), so a warp that finishes early takes
    // more tiles and the phase ends when the work, not the slowest warp's share,
    // is done.  Two counters alternate between phases; entering a phase, CTA 0
    // re-arms the other one, whose phase ended at the last grid barrier.  The
    // inner products are exact sums, so the order of tiles changes no result.
    constexpr bool dyn = DYN;
    int ph = 0;
    auto claim = [&](unsigned* c) -> int64_t {
        unsigned v = 0u;
        if (lane == 0) v = atomicAdd(c, 1u);
        return (int64_t)__shfl_sync(0xffffffffu, v, 0);
    };
    auto tiles_begin = [&](int64_t& t0, int64_t& t1, unsigned*& c) {
        if constexpr (dyn) {
            c = P.tilectr + ph;
            if (rank == 0 && threadIdx.x == 0) P.tilectr[ph ^ 1] = 0u;
            ph ^= 1;
            t0 = claim(c);
            t1 = claim(c);
        } else {
            c = nullptr;
            t0 = gwarp;
            t1 = gwarp + nwarps;
        }
    };
    // the tile after t1 (static: t1 + nwarps)
    auto tiles_next = [&](int64_t t1, unsigned* c) -> int64_t {
        if constexpr (dyn) return claim(c);
        else return t1 + nwarps;
    };
    // stage the warp's first two tiles of a phase (after the grid barrier that
    // made the previous phase's writes visible)
    auto stage_two = [&](auto first, const auto& v, int64_t t0, int64_t t1) {
        constexpr unsigned F = decltype(first)::value;
        if (t0 < ntiles) stg.template issue<F, kH>(v, t0, 0, polv);
        if (t1 < ntiles) stg.template issue<F, kH>(v, t1, 1, polv);
    };
    // after a tile's rows were read: refill its stage with tile t (two ahead)
    auto stage_at = [&](auto first, const auto& v, int64_t t, int64_t kt) {
        constexpr unsigned F = decltype(first)::value;
        if (t < ntiles) stg.template issue<F, kH>(v, t, (int)(kt & 1), polv);
    };
    // L2 policy of the row-local vector streams (see l2_first): a vector read or
    // written by a phase is marked evict_first when its next use is an
    // iteration away or when the phase overwrites it; the vectors that the next
    // phase reads stay at normal priority.  Staging masks per phase (bit k =
    // entry k of the phase's vector list).  Applied with FP32 vectors only
    // (l2_hints), and evict_first only when the solve's re-read set fits in L2
    // (KParams::l2hint; otherwise the same streams carry evict_normal).
    using FirstPA = std::integral_constant<unsigned, 0u>;                        // Y R RS
    using FirstPB = std::integral_constant<unsigned, 1u << 2>;                   // R s T Y P U
    using FirstPC = std::integral_constant<unsigned, 0xADu>;                     // O R U s Y P RS Z
    using FirstA = std::integral_constant<unsigned, 0x638u>;                     // R s RS P U T L Y G W Z
    using FirstC = std::integral_constant<unsigned, 0xFu>;                       // O L G s Y R RS

    auto st1 = [&](VT* p, VT v) {
        if constexpr (kH) st_first(p, v, polv);
        else *p = v;
    };
    auto ld1 = [&](const VT* p) -> VT {
        if constexpr (kH) return ld_first(p, polv);
        else return *p;
    };

    // ---- SELL: the solve runs in the permuted row order ----
    if (P.perm != nullptr) {
        for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
            const RowT row = (RowT)(tile * 32) + lane;
            if (row < n) {
                const int32_t src = __ldg(P.perm + row);
                P.x64[row] = P.x[src];
                P.b64w[row] = P.b[src];
            }
        }
        if (!grp.sync(&s_flag)) { stg.settle(); return; }
    }

    // ---- partitioned solve: this rank's rows of the caller's x (and their
    // copies in the other ranks' halos) ----
    if constexpr (DIST) {
        for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
            const RowT row = (RowT)(tile * 32) + lane;
            if (row < n) {
                const double xv = P.xg[P.row0 + row];
                P.x64[row] = xv;
                push(NVEC, tile, row, xv);
            }
        }
        if (!grp.sync(&s_flag)) { stg.settle(); return; }
    }

    int status = BCS_NOT_CONVERGED, inner_status = BCS_OK;
    int n_spmv = 0, n_red = 0;  // passes over the matrix and grid reductions (reported with the result)
    const unsigned long long t_start = global_ns();
    // barriers reported with the result: from here on; a partitioned solve
    // counts every barrier of the launch (its prologue's too), since the
    // one-process-per-GPU form continues the shared counter from that count
    if constexpr (!DIST) grp.nsync = 0;
    int total = 0, evals = 0, runs = 0, hist_len = 0, rr_steps = 0, fallbacks = 0;
    double r0n = 0.0, thresh = 0.0, r0ref = 1.0, rtrue = 0.0, last_rec = 0.0;
    double alpha_p = 0.0, zeta_p = 0.0, f_p = 0.0;  // thread 0 of each CTA
    double best_rn = 0.0;                            // refinement modes: stall guard (thread 0)
    int since_best = 0;

    for (;;) {
        if constexpr (BJ) {
            // the products of the true residual gather M^-1 y
            for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
                const RowT row = (RowT)(tile * 32) + lane;
                const double h = bj_apply(P.bj64, row < n ? P.x64[row] : 0.0, row);
                if (row < n) P.xhat64[row] = h;
            }
            if (!grp.sync(&s_flag)) { stg.settle(); return; }
        }
        // ---------------- true residual r = b - A x (FP64) and (re)initialisation ----------
        {
            typename DotAccOf<VT>::type xv[10];
            wa_init10(xv);
            WAcc xt[10];  // the FP64 true-residual norm is always accumulated exactly
            wa_init10(xt);
            for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
                const double ax = spmv64(BJ ? (const double*)P.xhat64 : P.x64, tile);
                const RowT row = (RowT)(tile * 32) + lane;
                double qa_ST = double(0), qb_ST = double(0);
                VT qa_SF = VT(0), qb_SF = VT(0);
                if (row < n) {
                    const double r64 = P.b64[row] - ax;
                    qa_ST = r64;
                    qb_ST = r64;
                    const VT rv = (VT)r64;
                    R[row] = rv;
                    push(V_R, tile, row, rv);
                    RS[row] = rv;
                    if (mixed) {
                        BinW[row] = rv;
                        X[row] = VT(0);
                    }
                    Y[row] = VT(0); Tv[row] = VT(0); Pv[row] = VT(0); U[row] = VT(0);
                    Z[row] = VT(0); W[row] = VT(0); L[row] = VT(0); G[row] = VT(0);
                    qa_SF = rv;
                    qb_SF = rv;
                }
                if constexpr (BJ) {   // qa_SF = r on the lane's row (0 beyond n)
                    const VT h = bj_apply(BJE, qa_SF, row);
                    if (row < n) RH[row] = h;
                }
                wa_acc(xt[ST], qa_ST, qb_ST, row < n, was);
                wa_acc(xv[SF], qa_SF, qb_SF, row < n, was);
            }
            xv[SR] = xv[SF];
            flush_partials<(1u << SF) | (1u << SR), (1u << SB) | (1u << SC) | (1u << SE) | (1u << SH)>(xv, s_x,
                                                                                                    myrec(0));
            flush_partials<(1u << ST)>(xt, s_x, myrec(0));
            if (!grp.sync(&s_flag)) { stg.settle(); return; }
            reduce_partials<10>(rbase(0), nblk, s_x, s_sum);
            ++n_spmv;
            ++n_red;
            const double rt2 = s_sum[ST];
            rtrue = sqrt(rt2);
            if (evals == 0) {
                r0n = rtrue;
                thresh = P.tol * r0n;
                r0ref = r0n > 0.0 ? r0n : 1.0;
            }
            ++evals;
            if (inner_status != BCS_OK) { status = inner_status; break; }
            if (rtrue <= thresh) { status = BCS_OK; break; }
            if (runs >= P.max_outer) { status = BCS_NOT_CONVERGED; break; }
        }
        ++runs;
        const double thr_in = mixed ? P.inner_tol * rtrue : thresh;
        const int budget = P.maxit - total;

        // ---------------- pipelined set-up: s_0 = A r_0 and the i = 0 products --------------
        if (kind != BCS_SSBICGSAFE2) {
            typename DotAccOf<VT>::type xv[10];
            wa_init10(xv);
            ++n_spmv;
            for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
                const VT sv = spmv(BJ ? RH : R, tile);
                const RowT row = (RowT)(tile * 32) + lane;
                if constexpr (BJ) {
                    const VT h = bj_apply(BJE, sv, row);
                    if (row < n) SHc[row] = h;
                }
                VT qa_SA = VT(0), qb_SA = VT(0);
                VT qa_SD = VT(0), qb_SD = VT(0);
                VT qa_SG = VT(0), qb_SG = VT(0);
                if (row < n) {
                    sCur[row] = sv;
                    push(sCurId, tile, row, sv);
                    const VT rv = R[row], rsv = RS[row];
                    qa_SA = sv;
                    qb_SA = sv;
                    qa_SD = sv;
                    qb_SD = rv;
                    qa_SG = rsv;
                    qb_SG = sv;
                }
                wa_acc(xv[SA], qa_SA, qb_SA, row < n, was);
                wa_acc(xv[SD], qa_SD, qb_SD, row < n, was);
                wa_acc(xv[SG], qa_SG, qb_SG, row < n, was);
            }
            flush_partials<(1u << SA) | (1u << SD) | (1u << SG)>(xv, s_x, myrec(0));
            if (!grp.sync(&s_flag)) { stg.settle(); return; }
        }

        // ---------------- iterations ----------------------------------------------------------
        int i = 0;
        for (;; ++i) {
            const int cur = i & 1, nxt = cur ^ 1;
            const bool rr_step = (kind == BCS_P_BICGSAFE_RR) && i > 0 && (i % P.rr_m) == 0 && i < P.rr_M;
            typename DotAccOf<VT>::type xv[10];
            VT as_first = VT(0);
            bool have_first = false;   // this warp's first-tile A s_i was formed during the reduction
            int64_t pa0 = 0, pa1 = 0;   // p-BiCGSafe phase A: the warp's first two tiles
            unsigned* pac = nullptr;
            if (kind == BCS_SSBICGSAFE2) {
                // phase A: s_i = A r_i and the products involving s_i
                wa_init10(xv);
                const VT* const vPA[] = {Y, R, RS};
                ++n_spmv;
                int64_t t0, t1;
                unsigned* tc;
                tiles_begin(t0, t1, tc);
                stage_two(FirstPA{}, vPA, t0, t1);
                int rpa = 0, rpb = 0;
                if (kRp) rp_load(t0, rpa, rpb);
                for (int64_t kt = 0; t0 < ntiles; ++kt) {
                    const int64_t tile = t0;
                    const int64_t t2 = tiles_next(t1, tc);
                    int rpa_n = 0, rpb_n = 0;
                    if (kRp) rp_load(t1, rpa_n, rpb_n);
                    const VT sv = spmv_rp(BJ ? RH : R, tile, rpa, rpb);
                    rpa = rpa_n; rpb = rpb_n;
                    const VT* sm = stg.wait((int)(kt & 1));
                    const RowT row = (RowT)(tile * 32) + lane;
                    VT qa_SA = VT(0), qb_SA = VT(0);
                    VT qa_SC = VT(0), qb_SC = VT(0);
                    VT qa_SD = VT(0), qb_SD = VT(0);
                    VT qa_SG = VT(0), qb_SG = VT(0);
                    if (row < n) {
                        sCur[row] = sv;
                        const VT yv = sm[lane], rv = sm[32 + lane], rsv = sm[64 + lane];
                        qa_SA = sv;
                        qb_SA = sv;
                        qa_SC = sv;
                        qb_SC = yv;
                        qa_SD = sv;
                        qb_SD = rv;
                        qa_SG = rsv;
                        qb_SG = sv;
                    }
                    wa_acc(xv[SA], qa_SA, qb_SA, row < n, was);
                    wa_acc(xv[SC], qa_SC, qb_SC, row < n, was);
                    wa_acc(xv[SD], qa_SD, qb_SD, row < n, was);
                    wa_acc(xv[SG], qa_SG, qb_SG, row < n, was);
                    stage_at(FirstPA{}, vPA, t2, kt);
                    t0 = t1;
                    t1 = t2;
                }
                flush_partials<(1u << SA) | (1u << SC) | (1u << SD) | (1u << SG)>(xv, s_x, myrec(cur));
                if (!grp.sync(&s_flag)) { stg.settle(); return; }
            } else {
                // phase A: A s_i of the first tile is in flight while the partials of
                // iteration i are reduced (the overlap of the reduction with MV, Section 3)
                if (!rr_step) {
                    // warps 1..9 reduce the nine slots while the others compute their
                    // first tile's A s_i (so the reduction runs under the SpMV's memory
                    // latency); warps 1..9 form their first tile's product in the tile
                    // loop, after the scalars (measured 3 % faster per iteration than
                    // forming it while warp 0 computes the scalars, which kept every
                    // warp waiting for those products at the scalars' barrier)
                    reduce_issue<9, NW, kRedOff>(rbase(cur), nblk);   // records travel to L1
                    const VT* const vA0[] = {R, sCur, RS, Pv, U, Tv, L, Y, G, W, Z};
                    tiles_begin(pa0, pa1, pac);
                    stage_two(FirstA{}, vA0, pa0, pa1);
                    const bool reducer = kRedOff > 0 && warp >= kRedOff && warp < kRedOff + 9;
                    have_first = !reducer && pa0 < ntiles;
                    if (have_first) as_first = spmv(BJ ? SHc : sCur, pa0);
                    reduce_finish<9, NW, kRedOff>(rbase(cur), nblk, s_x, s_sum);
                } else {
                    reduce_partials<9>(rbase(cur), nblk, s_x, s_sum);
                }
            }
            if (kind == BCS_SSBICGSAFE2) reduce_partials<9>(rbase(cur), nblk, s_x, s_sum);
            ++n_red;

            // ---- scalar recurrence and stop test (Alg. 3/4 i = 0 branch and general case) ----
            // The independent quotients are formed side by side by the lanes of
            // warp 0 (one division sequence) while warp kSqrtWarp takes the square
            // root; thread 0 then finishes alpha and the bookkeeping.  Every value is
            // the same IEEE quotient of the same operands as in a sequential
            // evaluation.
            if (warp == 0 && lane < 4) {
                const double a = s_sum[SA], bb = s_sum[SB], c = s_sum[SC], d = s_sum[SD], e = s_sum[SE];
                const double f = s_sum[SF], g = s_sum[SG];
                const double den = a * bb - c * c;
                double num = d, dv = a;  // lane 3: d / a
                if (lane == 0) {
                    num = i == 0 ? f : alpha_p * f;
                    dv = i == 0 ? g : zeta_p * f_p;
                } else if (lane == 1) {
                    num = bb * d - c * e;
                    dv = den;
                } else if (lane == 2) {
                    num = a * e - c * d;
                    dv = den;
                }
                s_q[lane] = num / dv;
            } else if (warp == kSqrtWarp && lane == 0) {
                s_q[4] = sqrt(s_sum[SR]);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const double a = s_sum[SA], bb = s_sum[SB], c = s_sum[SC];
                const double f = s_sum[SF], g = s_sum[SG], h = s_sum[SH], rr = s_sum[SR];
                double alpha, beta, zeta, eta;
                bool brk;
                if (i == 0) {
                    beta = 0.0;
                    alpha = s_q[0];   // f / g
                    zeta = s_q[3];    // d / a
                    eta = 0.0;
                    brk = (g == 0.0 || a == 0.0);
                } else {
                    beta = s_q[0];    // (alpha_{i-1} f_i) / (zeta_{i-1} f_{i-1})
                    alpha = f / (g + beta * h);
                    const double den = a * bb - c * c;
                    if (den == 0.0 || !isfinite(den)) {
                        zeta = s_q[3];
                        eta = 0.0;
                        ++fallbacks;
                    } else {
                        zeta = s_q[1];
                        eta = s_q[2];
                    }
                    brk = (zeta_p * f_p == 0.0 || g + beta * h == 0.0 || a == 0.0);
                }
                const double rn = s_q[4];
                const bool conv = rn <= thr_in;
                if (i == 0 || rn < best_rn) { best_rn = rn; since_best = 0; } else { ++since_best; }
                int dec = 0, st = BCS_OK;
                if (brk && !conv) {
                    dec = 1;
                    st = BCS_ERR_BREAKDOWN;
                } else {
                    if (writer) {
                        if (hist_len < P.hist_cap) P.hist[hist_len] = rn / r0ref;
                        if (runs == 1 && i < P.hist_cap) {
                            P.scal[4 * i + 0] = alpha; P.scal[4 * i + 1] = beta;
                            P.scal[4 * i + 2] = zeta;  P.scal[4 * i + 3] = eta;
                        }
                    }
                    ++hist_len;
                    last_rec = rn / r0ref;
                    if (conv) { dec = 1; st = BCS_OK; }
                    else if (!isfinite(alpha) || !isfinite(beta) || !isfinite(zeta) || !isfinite(eta) || !isfinite(rr)) {
                        dec = 1; st = BCS_ERR_NONFINITE;
                    } else if (i >= budget) { dec = 1; st = BCS_NOT_CONVERGED; }
                    else if (mixed && ((P.inner_maxit > 0 && i >= P.inner_maxit) ||
                                       (P.inner_stall > 0 && since_best >= P.inner_stall))) {
                        // low-precision inner run capped or no longer improving: hand
                        // back to the FP64 outer step (true residual, fresh Krylov space)
                        dec = 1; st = BCS_OK;
                    }
                }
                s_sc[0] = alpha; s_sc[1] = beta; s_sc[2] = zeta; s_sc[3] = eta;
                s_ctl[0] = dec; s_ctl[1] = st;
                alpha_p = alpha; zeta_p = zeta; f_p = f;
            }
            __syncthreads();
            if (s_ctl[0]) {
                // the run stops here: the staged first tiles of this phase A are not used
                stg.settle();
                inner_status = s_ctl[1];
                break;
            }
            const VT al = (VT)s_sc[0], be = (VT)s_sc[1], ze = (VT)s_sc[2], et = (VT)s_sc[3];

            if (kind == BCS_SSBICGSAFE2) {
                // phase B: p_i, o_i, u_i
                const VT* const vPB[] = {R, sCur, Tv, Y, Pv, U};
                int64_t b0, b1;
                unsigned* tb;
                tiles_begin(b0, b1, tb);
                stage_two(FirstPB{}, vPB, b0, b1);
                for (int64_t kt = 0; b0 < ntiles; ++kt) {
                    const int64_t tile = b0;
                    const int64_t b2 = tiles_next(b1, tb);
                    const VT* sm = stg.wait((int)(kt & 1));
                    const RowT row = (RowT)(tile * 32) + lane;
                    VT u_out = VT(0);
                    if (row < n) {
                        const VT r = sm[lane], s = sm[32 + lane], t = sm[64 + lane], y = sm[96 + lane];
                        VT p = sm[128 + lane], u = sm[160 + lane];
                        p = vfma(be, p - u, r);
                        const VT o = vfma(be, t, s);
                        u = vfma(ze, o, et * vfma(be, u, y));
                        Pv[row] = p; O[row] = o; U[row] = u;
                        push(V_U, tile, row, u);
                        u_out = u;
                    }
                    if constexpr (BJ) {
                        const VT h = bj_apply(BJE, u_out, row);
                        if (row < n) UH[row] = h;
                    }
                    (void)u_out;
                    stage_at(FirstPB{}, vPB, b2, kt);
                    b0 = b1;
                    b1 = b2;
                }
                if (!grp.sync(&s_flag)) { stg.settle(); return; }
                // phase C: w_i = A u_i; t_i, z_i, y_{i+1}, x_{i+1}, r_{i+1}
                wa_init10(xv);
                const VT* const vPC[] = {O, R, U, sCur, Y, Pv, RS, Z};
                ++n_spmv;
                int64_t c0, c1;
                unsigned* tcc;
                tiles_begin(c0, c1, tcc);
                stage_two(FirstPC{}, vPC, c0, c1);
                int rpa = 0, rpb = 0;
                if (kRp) rp_load(c0, rpa, rpb);
                for (int64_t kt = 0; c0 < ntiles; ++kt) {
                    const int64_t tile = c0;
                    const int64_t c2 = tiles_next(c1, tcc);
                    int rpa_n = 0, rpb_n = 0;
                    if (kRp) rp_load(c1, rpa_n, rpb_n);
                    const VT w = spmv_rp(BJ ? UH : U, tile, rpa, rpb);
                    rpa = rpa_n; rpb = rpb_n;
                    const VT* sm = stg.wait((int)(kt & 1));
                    const RowT row = (RowT)(tile * 32) + lane;
                    VT qa_SB = VT(0), qb_SB = VT(0);
                    VT qa_SE = VT(0), qb_SE = VT(0);
                    VT qa_SF = VT(0), qb_SF = VT(0);
                    VT qa_SH = VT(0), qb_SH = VT(0);
                    VT qa_SR = VT(0), qb_SR = VT(0);
                    if (row < n) {
                        const VT o = sm[lane], r = sm[32 + lane], u = sm[64 + lane], s = sm[96 + lane];
                        const VT y = sm[128 + lane], p = sm[160 + lane], rs = sm[192 + lane];
                        VT z = sm[224 + lane], x = ld1(X + row);
                        const VT t = o - w;
                        z = vfma(-al, u, vfma(ze, r, et * z));
                        const VT yn = vfma(-al, w, vfma(ze, s, et * y));
                        x = vfma(al, p, x) + z;
                        const VT rn = vfma(-al, o, r) - yn;
                        Tv[row] = t; st1(Z + row, z); Y[row] = yn; st1(X + row, x); R[row] = rn;
                        push(xId, tile, row, x);
                        push(V_R, tile, row, rn);
                        qa_SB = yn;
                        qb_SB = yn;
                        qa_SE = yn;
                        qb_SE = rn;
                        qa_SF = rs;
                        qb_SF = rn;
                        qa_SH = rs;
                        qb_SH = t;
                        qa_SR = rn;
                        qb_SR = rn;
                    }
                    wa_acc(xv[SB], qa_SB, qb_SB, row < n, was);
                    wa_acc(xv[SE], qa_SE, qb_SE, row < n, was);
                    wa_acc(xv[SF], qa_SF, qb_SF, row < n, was);
                    wa_acc(xv[SH], qa_SH, qb_SH, row < n, was);
                    wa_acc(xv[SR], qa_SR, qb_SR, row < n, was);
                    if constexpr (BJ) {   // qa_SR = r_{i+1} on the lane's row (0 beyond n)
                        const VT h = bj_apply(BJE, qa_SR, row);
                        if (row < n) RH[row] = h;
                    }
                    stage_at(FirstPC{}, vPC, c2, kt);
                    c0 = c1;
                    c1 = c2;
                }
                flush_partials<(1u << SB) | (1u << SE) | (1u << SF) | (1u << SH) | (1u << SR)>(xv, s_x, myrec(nxt));
                if (!grp.sync(&s_flag)) { stg.settle(); return; }
            } else if (!rr_step) {
                // phase A (continued): fused recurrences of Alg. 4
                ++n_spmv;  // A s_i (its first tile already above)
                wa_init10(xv);
                const VT* const vA[] = {R, sCur, RS, Pv, U, Tv, L, Y, G, W, Z};
                int rpa = 0, rpb = 0;
                if (kRp) rp_load(pa1, rpa, rpb);
                for (int64_t kt = 0; pa0 < ntiles; ++kt) {
                    const int64_t tile = pa0;
                    const int64_t pa2 = tiles_next(pa1, pac);
                    int rpa_n = 0, rpb_n = 0;
                    if (kRp && kt > 0) rp_load(pa1, rpa_n, rpb_n);
                    const VT* const sx = BJ ? SHc : sCur;
                    const VT As = (kt == 0) ? (have_first ? as_first : spmv(sx, tile)) : spmv_rp(sx, tile, rpa, rpb);
                    if (kt > 0) { rpa = rpa_n; rpb = rpb_n; }
                    const VT* sm = stg.wait((int)(kt & 1));
                    const RowT row = (RowT)(tile * 32) + lane;
                    VT qa_SB = VT(0), qb_SB = VT(0);
                    VT qa_SE = VT(0), qb_SE = VT(0);
                    VT qa_SF = VT(0), qb_SF = VT(0);
                    VT qa_SH = VT(0), qb_SH = VT(0);
                    VT qa_SR = VT(0), qb_SR = VT(0);
                    VT w_out = VT(0);
                    if (row < n) {
                        const VT r = sm[lane], s = sm[32 + lane], rs = sm[64 + lane];
                        VT p = sm[96 + lane], u = sm[128 + lane], t = sm[160 + lane], l = sm[192 + lane];
                        VT y = sm[224 + lane], g = sm[256 + lane], w = sm[288 + lane], z = sm[320 + lane];
                        VT x = ld1(X + row);
                        p = vfma(be, p - u, r);
                        const VT o = vfma(be, t, s);
                        u = vfma(ze, o, et * vfma(be, u, y));
                        const VT q = vfma(be, l, As);
                        w = vfma(ze, q, et * vfma(be, w, g));
                        t = o - w;
                        z = vfma(-al, u, vfma(ze, r, et * z));
                        const VT yn = vfma(-al, w, vfma(ze, s, et * y));
                        x = vfma(al, p, x) + z;
                        const VT rn = vfma(-al, o, r) - yn;
                        st1(Pv + row, p); st1(U + row, u); W[row] = w; st1(Tv + row, t); st1(Z + row, z);
                        w_out = w;
                        Y[row] = yn; st1(X + row, x); R[row] = rn; O[row] = As;
                        push(V_W, tile, row, w);
                        push(xId, tile, row, x);
                        qa_SB = yn;
                        qb_SB = yn;
                        qa_SE = yn;
                        qb_SE = rn;
                        qa_SF = rs;
                        qb_SF = rn;
                        qa_SH = rs;
                        qb_SH = t;
                        qa_SR = rn;
                        qb_SR = rn;
                    }
                    wa_acc(xv[SB], qa_SB, qb_SB, row < n, was);
                    wa_acc(xv[SE], qa_SE, qb_SE, row < n, was);
                    wa_acc(xv[SF], qa_SF, qb_SF, row < n, was);
                    wa_acc(xv[SH], qa_SH, qb_SH, row < n, was);
                    wa_acc(xv[SR], qa_SR, qb_SR, row < n, was);
                    if constexpr (BJ) {
                        const VT h = bj_apply(BJE, w_out, row);
                        if (row < n) WH[row] = h;
                    }
                    (void)w_out;
                    stage_at(FirstA{}, vA, pa2, kt);
                    pa0 = pa1;
                    pa1 = pa2;
                }
                flush_partials<(1u << SB) | (1u << SE) | (1u << SF) | (1u << SH) | (1u << SR)>(xv, s_x, myrec(nxt));
                if (!grp.sync(&s_flag)) { stg.settle(); return; }
                // phase C: A w_i; q_i (again), l_i, g_{i+1}, s_{i+1} and the products
                // involving s_{i+1}.  A s_i crosses the barrier in o (unused by this
                // method outside the replacement step), so that phase A stores one
                // vector instead of q, g' and s'; the expressions are the same.
                wa_init10(xv);
                const VT* const vC[] = {O, L, G, sCur, Y, R, RS};
                ++n_spmv;
                int64_t c0, c1;
                unsigned* tcc;
                tiles_begin(c0, c1, tcc);
                stage_two(FirstC{}, vC, c0, c1);
                rpa = 0; rpb = 0;
                if (kRp) rp_load(c0, rpa, rpb);
                for (int64_t kt = 0; c0 < ntiles; ++kt) {
                    const int64_t tile = c0;
                    const int64_t c2 = tiles_next(c1, tcc);
                    int rpa_n = 0, rpb_n = 0;
                    if (kRp) rp_load(c1, rpa_n, rpb_n);
                    const VT Aw = spmv_rp(BJ ? WH : W, tile, rpa, rpb);
                    rpa = rpa_n; rpb = rpb_n;
                    const VT* sm = stg.wait((int)(kt & 1));
                    const RowT row = (RowT)(tile * 32) + lane;
                    VT qa_SA = VT(0), qb_SA = VT(0);
                    VT qa_SC = VT(0), qb_SC = VT(0);
                    VT qa_SD = VT(0), qb_SD = VT(0);
                    VT qa_SG = VT(0), qb_SG = VT(0);
                    if (row < n) {
                        const VT As = sm[lane], lp = sm[32 + lane], gi = sm[64 + lane], si = sm[96 + lane];
                        const VT q = vfma(be, lp, As);
                        const VT gp = vfma(ze, As, et * gi);
                        const VT sa = vfma(-al, q, si);
                        const VT l = q - Aw;
                        const VT g = vfma(-al, Aw, gp);
                        const VT s = sa - g;
                        L[row] = l; G[row] = g; sNxt[row] = s;
                        push(sNxtId, tile, row, s);
                        const VT y = sm[128 + lane], r = sm[160 + lane], rs = sm[192 + lane];
                        qa_SA = s;
                        qb_SA = s;
                        qa_SC = s;
                        qb_SC = y;
                        qa_SD = s;
                        qb_SD = r;
                        qa_SG = rs;
                        qb_SG = s;
                    }
                    wa_acc(xv[SA], qa_SA, qb_SA, row < n, was);
                    wa_acc(xv[SC], qa_SC, qb_SC, row < n, was);
                    wa_acc(xv[SD], qa_SD, qb_SD, row < n, was);
                    wa_acc(xv[SG], qa_SG, qb_SG, row < n, was);
                    if constexpr (BJ) {   // qa_SA = s_{i+1} on the lane's row (0 beyond n)
                        const VT h = bj_apply(BJE, qa_SA, row);
                        if (row < n) SHn[row] = h;
                    }
                    stage_at(FirstC{}, vC, c2, kt);
                    c0 = c1;
                    c1 = c2;
                }
                flush_partials<(1u << SA) | (1u << SC) | (1u << SD) | (1u << SG)>(xv, s_x, myrec(nxt));
                if (!grp.sync(&s_flag)) { stg.settle(); return; }
                VT* tmp = sCur; sCur = sNxt; sNxt = tmp;
                const int tid = sCurId; sCurId = sNxtId; sNxtId = tid;
                if constexpr (BJ) { VT* th = SHc; SHc = SHn; SHn = th; }
            } else {
                // residual replacement iteration (Alg. 5)
                for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
                    const RowT row = (RowT)(tile * 32) + lane;
                    VT u_out = VT(0);
                    if (row < n) {
                        const VT r = R[row], s = sCur[row], t = Tv[row], y = Y[row];
                        VT p = Pv[row], u = U[row];
                        p = vfma(be, p - u, r);
                        const VT o = vfma(be, t, s);
                        u = vfma(ze, o, et * vfma(be, u, y));
                        Pv[row] = p; O[row] = o; U[row] = u;
                        push(V_U, tile, row, u);
                        u_out = u;
                    }
                    if constexpr (BJ) {
                        const VT h = bj_apply(BJE, u_out, row);
                        if (row < n) UH[row] = h;
                    }
                    (void)u_out;
                }
                if (!grp.sync(&s_flag)) { stg.settle(); return; }
                // w_i = A u_i (q_i = A o_i is not used after a replacement); t, z, y_{i+1}, x_{i+1}
                for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
                    const VT w = spmv(BJ ? UH : U, tile);
                    const RowT row = (RowT)(tile * 32) + lane;
                    VT t_out = VT(0), y_out = VT(0), x_out = VT(0);
                    if (row < n) {
                        const VT o = O[row], r = R[row], u = U[row], s = sCur[row], y = Y[row], p = Pv[row];
                        VT z = Z[row], x = X[row];
                        const VT t = o - w;
                        z = vfma(-al, u, vfma(ze, r, et * z));
                        const VT yn = vfma(-al, w, vfma(ze, s, et * y));
                        x = vfma(al, p, x) + z;
                        W[row] = w; Tv[row] = t; Z[row] = z; Y[row] = yn; X[row] = x;
                        push(xId, tile, row, x);
                        push(V_T, tile, row, t);
                        push(V_Y, tile, row, yn);
                        t_out = t; y_out = yn; x_out = x;
                    }
                    if constexpr (BJ) {
                        const VT ht = bj_apply(BJE, t_out, row);
                        const VT hy = bj_apply(BJE, y_out, row);
                        const VT hx = bj_apply(BJE, x_out, row);
                        if (row < n) { TH[row] = ht; YH[row] = hy; XH[row] = hx; }
                    }
                    (void)t_out; (void)y_out; (void)x_out;
                }
                if (!grp.sync(&s_flag)) { stg.settle(); return; }
                // r_{i+1} = b - A x_{i+1}; l_i = A t_i; g_{i+1} = A y_{i+1}
                wa_init10(xv);
                for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
                    const VT ax = spmv(BJ ? XH : X, tile);
                    const VT at = spmv(BJ ? TH : Tv, tile);
                    const VT ay = spmv(BJ ? YH : Y, tile);
                    const RowT row = (RowT)(tile * 32) + lane;
                    VT qa_SB = VT(0), qb_SB = VT(0);
                    VT qa_SE = VT(0), qb_SE = VT(0);
                    VT qa_SF = VT(0), qb_SF = VT(0);
                    VT qa_SH = VT(0), qb_SH = VT(0);
                    VT qa_SR = VT(0), qb_SR = VT(0);
                    if (row < n) {
                        const VT rn = Bin[row] - ax;
                        const VT y = Y[row], t = Tv[row], rs = RS[row];
                        R[row] = rn; L[row] = at; G[row] = ay;
                        push(V_R, tile, row, rn);
                        qa_SB = y;
                        qb_SB = y;
                        qa_SE = y;
                        qb_SE = rn;
                        qa_SF = rs;
                        qb_SF = rn;
                        qa_SH = rs;
                        qb_SH = t;
                        qa_SR = rn;
                        qb_SR = rn;
                    }
                    wa_acc(xv[SB], qa_SB, qb_SB, row < n, was);
                    wa_acc(xv[SE], qa_SE, qb_SE, row < n, was);
                    wa_acc(xv[SF], qa_SF, qb_SF, row < n, was);
                    wa_acc(xv[SH], qa_SH, qb_SH, row < n, was);
                    wa_acc(xv[SR], qa_SR, qb_SR, row < n, was);
                    if constexpr (BJ) {   // qa_SR = r_{i+1} on the lane's row (0 beyond n)
                        const VT h = bj_apply(BJE, qa_SR, row);
                        if (row < n) RH[row] = h;
                    }
                }
                flush_partials<(1u << SB) | (1u << SE) | (1u << SF) | (1u << SH) | (1u << SR)>(xv, s_x, myrec(nxt));
                if (!grp.sync(&s_flag)) { stg.settle(); return; }
                // s_{i+1} = A r_{i+1}
                wa_init10(xv);
                for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
                    const VT s = spmv(BJ ? RH : R, tile);
                    const RowT row = (RowT)(tile * 32) + lane;
                    if constexpr (BJ) {
                        const VT h = bj_apply(BJE, s, row);
                        if (row < n) SHn[row] = h;
                    }
                    VT qa_SA = VT(0), qb_SA = VT(0);
                    VT qa_SC = VT(0), qb_SC = VT(0);
                    VT qa_SD = VT(0), qb_SD = VT(0);
                    VT qa_SG = VT(0), qb_SG = VT(0);
                    if (row < n) {
                        sNxt[row] = s;
                        push(sNxtId, tile, row, s);
                        const VT y = Y[row], r = R[row], rs = RS[row];
                        qa_SA = s;
                        qb_SA = s;
                        qa_SC = s;
                        qb_SC = y;
                        qa_SD = s;
                        qb_SD = r;
                        qa_SG = rs;
                        qb_SG = s;
                    }
                    wa_acc(xv[SA], qa_SA, qb_SA, row < n, was);
                    wa_acc(xv[SC], qa_SC, qb_SC, row < n, was);
                    wa_acc(xv[SD], qa_SD, qb_SD, row < n, was);
                    wa_acc(xv[SG], qa_SG, qb_SG, row < n, was);
                }
                flush_partials<(1u << SA) | (1u << SC) | (1u << SD) | (1u << SG)>(xv, s_x, myrec(nxt));
                if (!grp.sync(&s_flag)) { stg.settle(); return; }
                ++rr_steps;
                n_spmv += 5;  // w = A u; A x, A t, A y; s = A r
                VT* tmp = sCur; sCur = sNxt; sNxt = tmp;
                if constexpr (BJ) { VT* th = SHc; SHc = SHn; SHn = th; }
                const int tid = sCurId; sCurId = sNxtId; sNxtId = tid;
            }
        }
        total += i;
        // refinement: x += d in FP64 (not after a non-finite inner run)
        if (mixed && inner_status != BCS_ERR_NONFINITE) {
            for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
                const RowT row = (RowT)(tile * 32) + lane;
                if (row < n) {
                    const double xn = P.x64[row] + (double)X[row];
                    P.x64[row] = xn;
                    push(NVEC, tile, row, xn);
                }
            }
        }
        if (!grp.sync(&s_flag)) { stg.settle(); return; }
    }

    if (writer && threadIdx.x == 0) {
        P.out[O_STATUS] = status;
        P.out[O_ITERS] = total;
        P.out[O_OUTER] = runs;
        P.out[O_RR] = rr_steps;
        P.out[O_FALLBACK] = fallbacks;
        P.out[O_RECREL] = last_rec;
        P.out[O_TRUEREL] = rtrue / r0ref;
        P.out[O_R0] = r0n;
        P.out[O_HISTLEN] = hist_len;
        P.out[O_SYNCS] = grp.nsync;
        P.out[O_REDUCTIONS] = n_red;
        P.out[O_SPMV] = n_spmv;
        P.out[O_T0] = (double)t_start;   // the system's start and end on the device clock (ns)
        P.out[O_T1] = (double)global_ns();
    }
    if (P.perm != nullptr) {
        for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
            const RowT row = (RowT)(tile * 32) + lane;
            if (row < n) P.x[__ldg(P.perm + row)] = P.x64[row];
        }
    }
    if constexpr (DIST) {
        for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
            const RowT row = (RowT)(tile * 32) + lane;
            if (row < n) P.xg[P.row0 + row] = P.x64[row];
        }
    }
}

template <class VT, class MT, int LAYOUT, int T, bool DYN, bool H = false, bool BJ = false, bool HI = false>
__global__ void __launch_bounds__(kSolveBlock, 1) solve_kernel(const __grid_constant__ KParams P) {
    GridGroup grp{GridBarrier{P.bar, P.err, gridDim.x, 0u, P.spin_budget}, (int)blockIdx.x, (int)gridDim.x};
    solve_body<VT, MT, LAYOUT, T, kSolveWarps, DYN, GridGroup, false, H, BJ, HI>(P, grp);
}

// Partitioned solve (bcs_dist.h): one cooperative launch whose CTAs are split
// into ranks; each CTA runs the solver body on its rank's row block, all CTAs
// meet at the one grid barrier and sum every rank's inner-product records.
template <class VT, class MT, bool SYS>
__global__ void __launch_bounds__(kSolveBlock, 1) solve_kernel_dist(const __grid_constant__ DistArgs D) {
    __shared__ KParams sP;
    __shared__ int s_r;
    if (threadIdx.x == 0) {
        int r = 0;
        while (r + 1 < D.nranks && (int)blockIdx.x >= D.cta0[r + 1]) ++r;
        s_r = r;
        sP = D.params[r];
    }
    __syncthreads();
    const int r = s_r;
    // records and barrier: this launch's CTAs are rec_offset .. of rec_total
    // (the CTAs of every process of the solve; all of them when one launch
    // holds every rank)
    GridGroupT<SYS> grp{GridBarrierT<SYS>{sP.bar, sP.err, (unsigned)D.rec_total, D.bar_base, sP.spin_budget},
                        D.rec_offset + (int)blockIdx.x, D.rec_total};
    grp.trank = (int)blockIdx.x - D.cta0[r];
    grp.tsize = D.cta0[r + 1] - D.cta0[r];
    solve_body<VT, MT, LAY_CSR, 1, kSolveWarps, false, GridGroupT<SYS>, true>(sP, grp);
}

// dynamic shared memory of the solver kernels: the per-warp staging buffers
template <class VT, int NW>
constexpr size_t stage_smem_bytes() {
    return (size_t)NW * 2 * kMaxStage * 32 * sizeof(VT);
}

template <class VT, class MT, int LAYOUT, int T, bool DYN, bool H = false, bool BJ = false, bool HI = false>
int launch_one(const KParams& P, int grid, cudaStream_t st) {
    void* args[] = {(void*)&P};
    const size_t smem = stage_smem_bytes<VT, kSolveWarps>();
    cudaError_t e = cudaFuncSetAttribute((const void*)solve_kernel<VT, MT, LAYOUT, T, DYN, H, BJ, HI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaLaunchCooperativeKernel((const void*)solve_kernel<VT, MT, LAYOUT, T, DYN, H, BJ, HI>, dim3(grid),
                                            dim3(kSolveBlock), args, smem, st);
}

template <class VT, class MT, int LAYOUT, int T, bool DYN, bool BJ = false>
int max_grid_one(int* grid) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = stage_smem_bytes<VT, kSolveWarps>();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)solve_kernel<VT, MT, LAYOUT, T, DYN, false, BJ>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, solve_kernel<VT, MT, LAYOUT, T, DYN, false, BJ>,
                                                          kSolveBlock, smem);
    *grid = sms * per;
    return (int)e;
}

// Partitioned solve of one (VT, MT) pair: launch (D != nullptr) or report the
// co-resident CTAs of the kernel (max_grid).
template <class VT, class MT>
int dispatch_dist(const DistArgs* D, int grid, cudaStream_t st, int* max_grid) {
    const size_t smem = stage_smem_bytes<VT, kSolveWarps>();
    const void* fn = (D && D->sys) ? (const void*)solve_kernel_dist<VT, MT, true>
                                   : (const void*)solve_kernel_dist<VT, MT, false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    if (!D) {
        int dev = 0, sms = 0, per = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, solve_kernel_dist<VT, MT, false>, kSolveBlock, smem);
        *max_grid = sms * per;
        return (int)e;
    }
    void* args[] = {(void*)D};
    return (int)cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kSolveBlock), args, smem, st);
}

// Dispatch over layout and lanes-per-row for one (VT, MT) pair; each
// translation unit instantiates one subset (SUBSET 0: SELL and CSR with 1 lane
// per row, SUBSET 1: CSR with 4, 8 or 32 lanes per row or adaptive (-1), both
// in the static tile order; SUBSET 2: the dynamic tile order for SELL and CSR
// with 1, 8 or adaptive lanes per row; SUBSET 3: block-Jacobi, CSR with 1
// lane per row in the static order).
template <class VT, class MT, int SUBSET>
int dispatch(const KParams* P, int layout, int tpr, int grid, cudaStream_t st, int* max_grid) {
#define BCS_CASE(LAY, TT, D)                                                              \
    return P ? launch_one<VT, MT, LAY, TT, D>(*P, grid, st) : max_grid_one<VT, MT, LAY, TT, D>(max_grid)
    if constexpr (SUBSET == 0) {
        if constexpr (sizeof(VT) == 8) {   // FP64 with the higher inner-product placement
            if (P && P->wa_hi) {
                if (layout == LAY_SELL) return launch_one<VT, MT, LAY_SELL, 1, false, false, false, true>(*P, grid, st);
                return launch_one<VT, MT, LAY_CSR, 1, false, false, false, true>(*P, grid, st);
            }
        }
        if (layout == LAY_SELL) { BCS_CASE(LAY_SELL, 1, false); }
        if constexpr (sizeof(VT) == 4) {   // CSR, one lane per row, with the L2 hints
            if (P && P->l2hint) return launch_one<VT, MT, LAY_CSR, 1, false, true>(*P, grid, st);
        }
        BCS_CASE(LAY_CSR, 1, false);
    } else if constexpr (SUBSET == 1) {
        switch (tpr) {
            case -1: BCS_CASE(LAY_CSR, 0, false);
            case 4: BCS_CASE(LAY_CSR, 4, false);
            case 8: BCS_CASE(LAY_CSR, 8, false);
            default: BCS_CASE(LAY_CSR, 32, false);
        }
    } else if constexpr (SUBSET == 3) {
        (void)layout;
        (void)tpr;
        return P ? launch_one<VT, MT, LAY_CSR, 1, false, false, true>(*P, grid, st)
                 : max_grid_one<VT, MT, LAY_CSR, 1, false, true>(max_grid);
    } else {
        if (layout == LAY_SELL) { BCS_CASE(LAY_SELL, 1, true); }
        if (tpr == 8) { BCS_CASE(LAY_CSR, 8, true); }
        if (tpr == -1) { BCS_CASE(LAY_CSR, 0, true); }
        BCS_CASE(LAY_CSR, 1, true);
    }
#undef BCS_CASE
}

}  // namespace bcs

namespace bcs {

__device__ __forceinline__ unsigned cluster_ctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_nctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_id_x() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

// Batched solves: each thread-block cluster takes systems from a work list
// (largest first) and solves them one after another with the same body as
// the single-system kernel; cluster barriers replace the grid barrier.
// sys[k]: the system's parameters without workspace; the cluster's own
// vectors (NVEC x max_n) and partials are patched in.


template <class VT, class MT, int T>
__global__ void __launch_bounds__(kBlock) batched_kernel(const __grid_constant__ BatchArgs B) {
    __shared__ KParams sP;
    __shared__ int s_dummy;
    ClusterGroup grp{(int)cluster_ctarank(), (int)cluster_nctarank()};
    const int cid = (int)cluster_id_x();
    for (;;) {
        if (grp.rank == 0 && threadIdx.x == 0) B.slots[cid] = atomicAdd(B.counter, 1);
        grp.sync(&s_dummy);
        const int k = ld_relaxed_int(B.slots + cid);
        grp.sync(&s_dummy);
        if (k >= B.nsys) break;
        if (threadIdx.x == 0) {
            sP = B.sys[B.order[k]];
            char* base = B.ws + (size_t)cid * B.ws_group_bytes;
            for (int v = 0; v < NVEC; ++v) sP.vec[v] = base + (size_t)v * B.vec_bytes;
            sP.partials = B.partials + (size_t)cid * 2 * B.csize * NSLOT * kRec;
        }
        __syncthreads();
        solve_body<VT, MT, LAY_CSR, T, kWarps, false>(sP, grp);
    }
}

template <class VT, class MT>
int dispatch_batched(const BatchArgs* B, int tpr, int nclusters, cudaStream_t st, int* max_clusters) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = B->csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = stage_smem_bytes<VT, kWarps>();
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void (*fn)(BatchArgs) = (tpr == 1) ? batched_kernel<VT, MT, 1> : batched_kernel<VT, MT, 8>;
    cudaError_t e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)stage_smem_bytes<VT, kWarps>());
    if (e == cudaSuccess && B->csize > 8)
        e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
    if (max_clusters) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cfg.gridDim = dim3(B->csize * sms);
        int mc = 0;
        e = cudaOccupancyMaxActiveClusters(&mc, (const void*)fn, &cfg);
        *max_clusters = mc;
        return (int)e;
    }
    cfg.gridDim = dim3(B->csize * nclusters);
    return (int)cudaLaunchKernelEx(&cfg, fn, *B);
}

}  // namespace bcs
