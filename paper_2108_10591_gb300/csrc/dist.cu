// Row-partitioned solve (include/bcs_dist.h): the partition, the halo plans
// and the C ABI of the solver whose ranks are CTA groups of one launch.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "bcs_dist.h"
#include "solver.cuh"

using namespace bcs;

namespace bcs {
int dispatch_dist_f64(const DistArgs* D, int grid, cudaStream_t st, int* max_grid);
int dispatch_dist_f32(const DistArgs* D, int grid, cudaStream_t st, int* max_grid);
int dispatch_dist_bf16(const DistArgs* D, int grid, cudaStream_t st, int* max_grid);
int options_check(const bcs_options& o);
long long spin_cycles(double ms);
int convert_values(const double* in, int valtype, void* out, int64_t m, cudaStream_t st);
}  // namespace bcs

namespace {

int64_t round32(int64_t v) { return ((v + 31) / 32) * 32; }

// One rank's block, halo and send list (global columns in left/right).
struct RankPlan {
    int64_t row0 = 0, nloc = 0, npad = 0;
    std::vector<int64_t> left, right;
    std::vector<int32_t> lcol;
    std::vector<int32_t> send_row, send_rank;
    std::vector<int64_t> send_off;
};

bool rowptr_ok(int64_t n, const int64_t* rowptr) {
    if (rowptr[0] != 0) return false;
    for (int64_t r = 0; r < n; ++r)
        if (rowptr[r + 1] < rowptr[r]) return false;
    return true;
}

bool bounds_ok(int64_t n, int nparts, const int64_t* bounds) {
    if (bounds[0] != 0 || bounds[nparts] != n) return false;
    for (int k = 0; k < nparts; ++k)
        if (bounds[k + 1] < bounds[k]) return false;
    return true;
}

// Offset of global column c in the offset space of rank q (c outside q's rows).
int64_t halo_offset(const RankPlan& q, int64_t c) {
    if (c < q.row0) {
        const int64_t k = std::lower_bound(q.left.begin(), q.left.end(), c) - q.left.begin();
        return k - (int64_t)q.left.size();
    }
    const int64_t k = std::lower_bound(q.right.begin(), q.right.end(), c) - q.right.begin();
    return q.npad + k;
}

// Every rank's plan (each rank's send list needs the other ranks' halos).
int make_plans(int64_t n, const int64_t* rowptr, const int32_t* col, int nparts, const int64_t* bounds,
               bool with_cols, std::vector<RankPlan>& plans) {
    plans.assign(nparts, RankPlan());
    for (int r = 0; r < nparts; ++r) {
        RankPlan& p = plans[r];
        p.row0 = bounds[r];
        p.nloc = bounds[r + 1] - bounds[r];
        p.npad = round32(p.nloc);
        const int64_t r1 = bounds[r + 1];
        for (int64_t k = rowptr[p.row0]; k < rowptr[r1]; ++k) {
            const int64_t c = col[k];
            if (c < p.row0) p.left.push_back(c);
            else if (c >= r1) p.right.push_back(c);
        }
        for (std::vector<int64_t>* v : {&p.left, &p.right}) {
            std::sort(v->begin(), v->end());
            v->erase(std::unique(v->begin(), v->end()), v->end());
        }
        if (p.npad + (int64_t)p.right.size() >= (int64_t)INT32_MAX) return BCS_ERR_ARG;
        if (with_cols) {
            p.lcol.resize((size_t)(rowptr[r1] - rowptr[p.row0]));
            for (int64_t k = rowptr[p.row0]; k < rowptr[r1]; ++k) {
                const int64_t c = col[k];
                const int64_t o = (c >= p.row0 && c < r1) ? c - p.row0 : halo_offset(p, c);
                p.lcol[(size_t)(k - rowptr[p.row0])] = (int32_t)o;
            }
        }
    }
    // send lists: rank q's halo column c is owned by the rank p whose block holds it
    struct Entry { int32_t row, rank; int64_t off; };
    std::vector<std::vector<Entry>> sends(nparts);
    for (int q = 0; q < nparts; ++q) {
        const RankPlan& pq = plans[q];
        for (const std::vector<int64_t>* v : {&pq.left, &pq.right}) {
            for (int64_t c : *v) {
                const int p = (int)(std::upper_bound(bounds, bounds + nparts + 1, c) - bounds) - 1;
                sends[p].push_back(Entry{(int32_t)(c - plans[p].row0), (int32_t)q, halo_offset(pq, c)});
            }
        }
    }
    for (int p = 0; p < nparts; ++p) {
        std::vector<Entry>& e = sends[p];
        std::sort(e.begin(), e.end(), [](const Entry& a, const Entry& b) {
            return a.row != b.row ? a.row < b.row : a.rank < b.rank;
        });
        for (const Entry& x : e) {
            plans[p].send_row.push_back(x.row);
            plans[p].send_rank.push_back(x.rank);
            plans[p].send_off.push_back(x.off);
        }
    }
    return BCS_OK;
}

bool csr_ok(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col) {
    if (!rowptr_ok(n, rowptr) || rowptr[n] != nnz) return false;
    for (int64_t r = 0; r < n; ++r)
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
            if (col[k] < 0 || col[k] >= n) return false;
            if (k > rowptr[r] && col[k] <= col[k - 1]) return false;
        }
    return true;
}

}  // namespace

extern "C" int bcs_partition_rows(int64_t n, const int64_t* rowptr, int nparts, int64_t* bounds) {
    if (n < 0 || !rowptr || !bounds || nparts < 1 || nparts > BCS_DIST_MAX_RANKS) return BCS_ERR_ARG;
    if (!rowptr_ok(n, rowptr)) return BCS_ERR_ARG;
    // weight of rows [0, r): rowptr[r] + r; block k ends at the row whose
    // prefix weight is nearest to k/nparts of the total
    const double total = (double)(rowptr[n] + n);
    bounds[0] = 0;
    int64_t lo = 0;
    for (int k = 1; k < nparts; ++k) {
        const double target = total * k / nparts;
        int64_t a = lo, b = n;   // first r in [lo, n] with weight(r) >= target
        while (a < b) {
            const int64_t m = a + (b - a) / 2;
            if ((double)(rowptr[m] + m) < target) a = m + 1; else b = m;
        }
        if (a > lo && target - (double)(rowptr[a - 1] + a - 1) < (double)(rowptr[a] + a) - target) --a;
        bounds[k] = a;
        lo = a;
    }
    bounds[nparts] = n;
    return BCS_OK;
}

extern "C" int bcs_halo_plan(int64_t n, const int64_t* rowptr, const int32_t* col, int nparts, const int64_t* bounds,
                             int rank, int64_t* nleft, int64_t* nright, int64_t* nsend, int32_t* local_col,
                             int64_t* left_cols, int64_t* right_cols, int32_t* send_row, int32_t* send_rank,
                             int64_t* send_off) {
    if (n < 0 || !rowptr || (rowptr[n] > 0 && !col) || !bounds || nparts < 1 || nparts > BCS_DIST_MAX_RANKS ||
        rank < 0 || rank >= nparts)
        return BCS_ERR_ARG;
    if (!csr_ok(n, rowptr[n], rowptr, col) || !bounds_ok(n, nparts, bounds)) return BCS_ERR_ARG;
    std::vector<RankPlan> plans;
    int rc;
    try {
        rc = make_plans(n, rowptr, col, nparts, bounds, local_col != nullptr, plans);
    } catch (const std::bad_alloc&) {
        return BCS_ERR_OOM;
    }
    if (rc) return rc;
    const RankPlan& p = plans[rank];
    if (nleft) *nleft = (int64_t)p.left.size();
    if (nright) *nright = (int64_t)p.right.size();
    if (nsend) *nsend = (int64_t)p.send_row.size();
    if (local_col && !p.lcol.empty()) memcpy(local_col, p.lcol.data(), p.lcol.size() * sizeof(int32_t));
    if (left_cols && !p.left.empty()) memcpy(left_cols, p.left.data(), p.left.size() * sizeof(int64_t));
    if (right_cols && !p.right.empty()) memcpy(right_cols, p.right.data(), p.right.size() * sizeof(int64_t));
    const size_t ns = p.send_row.size();
    if (send_row && ns) memcpy(send_row, p.send_row.data(), ns * sizeof(int32_t));
    if (send_rank && ns) memcpy(send_rank, p.send_rank.data(), ns * sizeof(int32_t));
    if (send_off && ns) memcpy(send_off, p.send_off.data(), ns * sizeof(int64_t));
    return BCS_OK;
}

// ---- the partitioned solver ---------------------------------------------------------------

struct bcs_dist_s {
    int nranks = 0, kind = 0, maxit = 0;
    double tol = 0;
    bcs_options opt;
    int vt_f32 = 0, valtype = VAL_F64, grid = 0;
    size_t vbytes = 8;
    int64_t n = 0;
    struct Rank {
        int64_t row0 = 0, nloc = 0, npad = 0, nleft = 0, nright = 0, nsend = 0, len = 0;
        int ctas = 0;
        int32_t* rowptr = nullptr;
        int32_t* col = nullptr;
        double* val64 = nullptr;
        void* valin = nullptr;        // FP32 / BF16 values (refinement modes)
        int32_t* send_ptr = nullptr;
        int2* send_dst = nullptr;
        unsigned char* tile_send = nullptr;
        char* vecmem = nullptr;       // NVEC vectors of len elements (halo included)
        double* x64 = nullptr;        // len doubles
    };
    std::vector<Rank> ranks;
    void** dpeer = nullptr;           // [nranks][NVEC + 1]
    KParams* dparams = nullptr;
    KParams* hparams = nullptr;       // pinned
    double* partials = nullptr;
    unsigned* bar = nullptr;
    double* hist = nullptr;
    double* scal = nullptr;
    double* out = nullptr;
    double* host_out = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int hist_len = 0;
    // one rank per process and GPU (bcs_dist_rank_create): this process holds
    // rank `rank` only; every rank's vectors, x, records and barrier counter
    // live in one arena per rank that the others open by CUDA IPC
    int proc = 0, rank = 0, total_ctas = 0, connected = 0;
    std::vector<int64_t> all_len, all_nleft;  // every rank's extended vector length and left halo
    char* arena = nullptr;
    std::vector<void*> opened;                // peers' arenas (IPC), nullptr for this rank
    double* rec = nullptr;                    // rank 0's records (all ranks write and read them)
    unsigned bar_base = 0;                    // barriers already passed on that counter
};

namespace {

// Arena of one rank in process mode: NVEC extended vectors, the FP64 x, the
// double-buffered records of every CTA of the solve, the barrier word; each
// part 256-byte aligned.  Every rank computes every rank's layout.
struct ArenaLayout {
    size_t vec, x64, rec, bar, bytes;
};
ArenaLayout arena_layout(int64_t len, size_t vbytes, int total_ctas) {
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    ArenaLayout a;
    a.vec = 0;
    a.x64 = up((size_t)NVEC * (size_t)len * vbytes);
    a.rec = a.x64 + up(sizeof(double) * (size_t)len);
    a.bar = a.rec + up(sizeof(double) * 2 * (size_t)total_ctas * NSLOT * kRec);
    a.bytes = a.bar + 256;
    return a;
}

int dist_dispatch(const bcs_dist_s* d, const DistArgs* D, int grid, cudaStream_t st, int* mg) {
    if (!d->vt_f32) return dispatch_dist_f64(D, grid, st, mg);
    if (d->valtype == VAL_F32) return dispatch_dist_f32(D, grid, st, mg);
    return dispatch_dist_bf16(D, grid, st, mg);
}

}  // namespace

extern "C" {

void bcs_dist_destroy(bcs_dist d) {
    if (!d) return;
    cudaDeviceSynchronize();
    for (auto& r : d->ranks) {
        if (d->proc) r.vecmem = nullptr, r.x64 = nullptr;   // parts of the arena
        void* ptrs[] = {r.rowptr, r.col, r.val64, r.valin, r.send_ptr, r.send_dst, r.tile_send, r.vecmem, r.x64};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    }
    if (d->proc) d->bar = nullptr;   // rank 0's barrier word, inside an arena
    for (void* p : d->opened)
        if (p) cudaIpcCloseMemHandle(p);
    if (d->arena) cudaFree(d->arena);
    void* ptrs[] = {d->dpeer, d->dparams, d->partials, d->bar, d->hist, d->scal, d->out};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (d->hparams) cudaFreeHost(d->hparams);
    if (d->host_out) cudaFreeHost(d->host_out);
    if (d->ev0) cudaEventDestroy(d->ev0);
    if (d->ev1) cudaEventDestroy(d->ev1);
    delete d;
}

}  // extern "C"

// Both forms of the partitioned solver: every rank in one launch on this GPU
// (proc_rank < 0), or rank proc_rank of a solve with one process per GPU.
static int dist_build(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col, const double* val,
                      int nparts, const int64_t* bounds, int proc_rank, int kind, double tol, int maxit,
                      const bcs_options* opt, bcs_dist* out) {
    if (!out) return BCS_ERR_ARG;
    *out = nullptr;
    if (n < 1 || n >= INT32_MAX || nnz < 0 || nnz >= INT32_MAX || !rowptr || (nnz > 0 && (!col || !val)) ||
        nparts < 1 || nparts > BCS_DIST_MAX_RANKS || kind < BCS_SSBICGSAFE2 || kind > BCS_P_BICGSAFE_RR ||
        !(tol >= 0.0) || maxit < 0)
        return BCS_ERR_ARG;
    bcs_options o;
    if (opt) o = *opt; else bcs_options_default(&o);
    if (o.rr_M == 0) o.rr_M = maxit < INT32_MAX ? maxit + 1 : maxit;
    if (options_check(o) != BCS_OK) return BCS_ERR_ARG;
    // one lane per CSR row, static tile order, no preconditioner
    if ((o.layout != BCS_LAYOUT_AUTO && o.layout != BCS_LAYOUT_CSR) || (o.threads_per_row != 0 && o.threads_per_row != 1) ||
        o.tile_order == 2 || o.precond != BCS_PRECOND_NONE)
        return BCS_ERR_ARG;
    if (!csr_ok(n, nnz, rowptr, col)) return BCS_ERR_ARG;
    std::vector<int64_t> bnd(nparts + 1);
    if (bounds) {
        if (!bounds_ok(n, nparts, bounds)) return BCS_ERR_ARG;
        std::copy(bounds, bounds + nparts + 1, bnd.begin());
    } else if (bcs_partition_rows(n, rowptr, nparts, bnd.data()) != BCS_OK) {
        return BCS_ERR_ARG;
    }
    std::vector<RankPlan> plans;
    int rc;
    try {
        rc = make_plans(n, rowptr, col, nparts, bnd.data(), true, plans);
    } catch (const std::bad_alloc&) {
        return BCS_ERR_OOM;
    }
    if (rc) return rc;

    bcs_dist d = new bcs_dist_s();
    d->nranks = nparts;
    d->kind = kind;
    d->tol = tol;
    d->maxit = maxit;
    d->opt = o;
    d->n = n;
    d->vt_f32 = o.precision != BCS_FP64;
    d->valtype = o.precision == BCS_FP64 ? VAL_F64 : o.precision == BCS_FP32_REFINE ? VAL_F32 : VAL_BF16;
    d->vbytes = d->vt_f32 ? sizeof(float) : sizeof(double);
    d->proc = proc_rank >= 0;
    d->rank = d->proc ? proc_rank : 0;
    const int r_lo = d->proc ? proc_rank : 0, r_hi = d->proc ? proc_rank + 1 : nparts;   // ranks held here
    d->ranks.resize(r_hi - r_lo);
    for (const RankPlan& p : plans) {
        const int64_t len = (int64_t)p.left.size() + std::max<int64_t>(p.npad, 32) + (int64_t)p.right.size();
        d->all_len.push_back(len);
        d->all_nleft.push_back((int64_t)p.left.size());
    }
    // CTAs: all co-resident ones, shared in proportion to the ranks' rows; one
    // process per GPU: all of this GPU's (the GPUs are taken to be alike)
    int maxg = 0;
    if (dist_dispatch(d, nullptr, 0, 0, &maxg) != 0 || maxg < (d->proc ? 1 : nparts)) {
        bcs_dist_destroy(d);
        return maxg > 0 ? BCS_ERR_ARG : BCS_ERR_CUDA;
    }
    if (d->proc) {
        d->ranks[0].ctas = maxg;
        d->grid = maxg;
        d->total_ctas = maxg * nparts;
    } else {
        int given = 0;
        for (int r = 0; r < nparts; ++r) {
            const int64_t want = (int64_t)((double)maxg * (double)plans[r].nloc / (double)n);
            d->ranks[r].ctas = (int)std::max<int64_t>(1, want);
            given += d->ranks[r].ctas;
        }
        for (int r = 0; given > maxg; r = (r + 1) % nparts)
            if (d->ranks[r].ctas > 1) { --d->ranks[r].ctas; --given; }
        d->grid = given;
        d->total_ctas = given;
    }
    for (int r = r_lo; r < r_hi; ++r) {
        const int64_t tiles = (plans[r].nloc + 31) / 32, warps = (int64_t)d->ranks[r - r_lo].ctas * kSolveWarps;
        if ((tiles + warps - 1) / warps >= (1 << 16)) {  // per-lane exact partials hold < 2^16 tiles
            bcs_dist_destroy(d);
            return BCS_ERR_ARG;
        }
    }
    rc = BCS_OK;
    auto alloc = [&](void** p, size_t bytes) {
        if (rc) return;
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) rc = BCS_ERR_OOM;
    };
    auto put = [&](void* dst, const void* src, size_t bytes) {
        if (rc || bytes == 0) return;
        if (cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) rc = BCS_ERR_CUDA;
    };
    std::vector<void*> peer((size_t)nparts * (NVEC + 1), nullptr);
    const ArenaLayout lay = arena_layout(d->all_len[d->rank], d->vbytes, d->total_ctas);
    if (d->proc) {
        alloc((void**)&d->arena, lay.bytes);
        if (!rc && cudaMemset(d->arena, 0, lay.bytes) != cudaSuccess) rc = BCS_ERR_CUDA;
    }
    for (int r = r_lo; r < r_hi && !rc; ++r) {
        const RankPlan& p = plans[r];
        bcs_dist_s::Rank& R = d->ranks[r - r_lo];
        R.row0 = p.row0;
        R.nloc = p.nloc;
        R.npad = std::max<int64_t>(p.npad, 32);
        R.nleft = (int64_t)p.left.size();
        R.nright = (int64_t)p.right.size();
        R.nsend = (int64_t)p.send_row.size();
        R.len = R.nleft + R.npad + R.nright;
        const int64_t k0 = rowptr[p.row0], nz = rowptr[p.row0 + p.nloc] - k0;
        std::vector<int32_t> rp((size_t)p.nloc + 1);
        for (int64_t i = 0; i <= p.nloc; ++i) rp[(size_t)i] = (int32_t)(rowptr[p.row0 + i] - k0);
        std::vector<int32_t> sp((size_t)p.nloc + 1, 0);
        std::vector<int2> sd((size_t)R.nsend);
        const int64_t ntiles = (p.nloc + 31) / 32;
        std::vector<unsigned char> ts((size_t)std::max<int64_t>(ntiles, 1), 0);
        for (int64_t k = 0; k < R.nsend; ++k) {
            sp[(size_t)p.send_row[(size_t)k] + 1]++;
            sd[(size_t)k] = make_int2(p.send_rank[(size_t)k], (int)p.send_off[(size_t)k]);
            ts[(size_t)(p.send_row[(size_t)k] / 32)] = 1;
        }
        for (int64_t i = 0; i < p.nloc; ++i) sp[(size_t)i + 1] += sp[(size_t)i];
        alloc((void**)&R.rowptr, sizeof(int32_t) * rp.size());
        alloc((void**)&R.col, sizeof(int32_t) * (size_t)nz);
        alloc((void**)&R.val64, sizeof(double) * (size_t)nz);
        if (d->vt_f32) alloc(&R.valin, (d->valtype == VAL_F32 ? sizeof(float) : sizeof(uint16_t)) * (size_t)nz);
        alloc((void**)&R.send_ptr, sizeof(int32_t) * sp.size());
        alloc((void**)&R.send_dst, sizeof(int2) * (size_t)R.nsend);
        alloc((void**)&R.tile_send, ts.size());
        if (d->proc) {
            R.vecmem = d->arena + lay.vec;
            R.x64 = (double*)(d->arena + lay.x64);
        } else {
            alloc((void**)&R.vecmem, (size_t)NVEC * (size_t)R.len * d->vbytes);
            alloc((void**)&R.x64, sizeof(double) * (size_t)R.len);
        }
        put(R.rowptr, rp.data(), sizeof(int32_t) * rp.size());
        put(R.col, p.lcol.data(), sizeof(int32_t) * (size_t)nz);
        put(R.val64, val + k0, sizeof(double) * (size_t)nz);
        put(R.send_ptr, sp.data(), sizeof(int32_t) * sp.size());
        put(R.send_dst, sd.data(), sizeof(int2) * (size_t)R.nsend);
        put(R.tile_send, ts.data(), ts.size());
        if (!rc && d->vt_f32 && nz > 0 && convert_values(R.val64, d->valtype, R.valin, nz, 0) != 0) rc = BCS_ERR_CUDA;
        if (!rc && cudaMemset(R.vecmem, 0, (size_t)NVEC * (size_t)R.len * d->vbytes) != cudaSuccess) rc = BCS_ERR_CUDA;
        if (!rc && cudaMemset(R.x64, 0, sizeof(double) * (size_t)R.len) != cudaSuccess) rc = BCS_ERR_CUDA;
        if (!rc) {
            for (int v = 0; v < NVEC; ++v)
                peer[(size_t)r * (NVEC + 1) + v] = R.vecmem + ((size_t)v * (size_t)R.len + (size_t)R.nleft) * d->vbytes;
            peer[(size_t)r * (NVEC + 1) + NVEC] = R.x64 + R.nleft;
        }
    }
    const size_t nrec = sizeof(double) * 2 * (size_t)d->grid * NSLOT * kRec;
    alloc((void**)&d->dpeer, sizeof(void*) * peer.size());
    if (!d->proc) put(d->dpeer, peer.data(), sizeof(void*) * peer.size());   // process mode: at connect
    alloc((void**)&d->dparams, sizeof(KParams) * (size_t)nparts);
    if (!d->proc) {
        alloc((void**)&d->partials, nrec);
        alloc((void**)&d->bar, 64);
    }
    alloc((void**)&d->hist, sizeof(double) * std::max(o.history_len, 1));
    alloc((void**)&d->scal, sizeof(double) * 4 * std::max(o.history_len, 1));
    alloc((void**)&d->out, sizeof(double) * NOUT);
    if (!rc && cudaMallocHost((void**)&d->host_out, sizeof(double) * NOUT + 64) != cudaSuccess) rc = BCS_ERR_OOM;
    if (!rc && cudaMallocHost((void**)&d->hparams, sizeof(KParams) * (size_t)nparts) != cudaSuccess) rc = BCS_ERR_OOM;
    if (!rc && (cudaEventCreate(&d->ev0) != cudaSuccess || cudaEventCreate(&d->ev1) != cudaSuccess)) rc = BCS_ERR_CUDA;
    if (!rc && !d->proc && cudaMemset(d->partials, 0, nrec) != cudaSuccess) rc = BCS_ERR_CUDA;
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = BCS_ERR_CUDA;
    if (rc) {
        bcs_dist_destroy(d);
        return rc;
    }
    *out = d;
    return BCS_OK;
}

extern "C" {

int bcs_dist_create(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col, const double* val,
                    int nparts, const int64_t* bounds, int kind, double tol, int maxit, const bcs_options* opt,
                    bcs_dist* out) {
    return dist_build(n, nnz, rowptr, col, val, nparts, bounds, -1, kind, tol, maxit, opt, out);
}

int bcs_dist_rank_create(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col, const double* val,
                         int nparts, const int64_t* bounds, int rank, int kind, double tol, int maxit,
                         const bcs_options* opt, bcs_dist* out) {
    if (rank < 0 || rank >= nparts) return BCS_ERR_ARG;
    return dist_build(n, nnz, rowptr, col, val, nparts, bounds, rank, kind, tol, maxit, opt, out);
}

int bcs_dist_rank_export(bcs_dist d, void* handle) {
    if (!d || !d->proc || !handle) return BCS_ERR_ARG;
    cudaIpcMemHandle_t h;
    if (cudaIpcGetMemHandle(&h, d->arena) != cudaSuccess) return BCS_ERR_CUDA;
    static_assert(sizeof(h) <= BCS_DIST_HANDLE_BYTES, "handle size");
    memset(handle, 0, BCS_DIST_HANDLE_BYTES);
    memcpy(handle, &h, sizeof(h));
    return BCS_OK;
}

int bcs_dist_rank_connect(bcs_dist d, const void* handles) {
    if (!d || !d->proc || !handles || d->connected) return BCS_ERR_ARG;
    const int P = d->nranks;
    d->opened.assign(P, nullptr);
    std::vector<char*> base(P, nullptr);
    for (int q = 0; q < P; ++q) {
        if (q == d->rank) {
            base[q] = d->arena;
            continue;
        }
        cudaIpcMemHandle_t h;
        memcpy(&h, (const char*)handles + (size_t)q * BCS_DIST_HANDLE_BYTES, sizeof(h));
        void* p = nullptr;
        if (cudaIpcOpenMemHandle(&p, h, cudaIpcMemLazyEnablePeerAccess) != cudaSuccess) return BCS_ERR_CUDA;
        d->opened[q] = p;
        base[q] = (char*)p;
    }
    std::vector<void*> peer((size_t)P * (NVEC + 1), nullptr);
    for (int q = 0; q < P; ++q) {
        const ArenaLayout lq = arena_layout(d->all_len[q], d->vbytes, d->total_ctas);
        for (int v = 0; v < NVEC; ++v)
            peer[(size_t)q * (NVEC + 1) + v] =
                base[q] + lq.vec + ((size_t)v * (size_t)d->all_len[q] + (size_t)d->all_nleft[q]) * d->vbytes;
        peer[(size_t)q * (NVEC + 1) + NVEC] = base[q] + lq.x64 + (size_t)d->all_nleft[q] * sizeof(double);
    }
    const ArenaLayout l0 = arena_layout(d->all_len[0], d->vbytes, d->total_ctas);
    d->rec = (double*)(base[0] + l0.rec);
    d->bar = (unsigned*)(base[0] + l0.bar);   // rank 0's barrier counter and error word
    if (cudaMemcpy(d->dpeer, peer.data(), sizeof(void*) * peer.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return BCS_ERR_CUDA;
    d->connected = 1;
    return BCS_OK;
}

int bcs_dist_solve(bcs_dist d, const double* b_dev, double* x_dev, bcs_result* res, void* stream) {
    NvtxRange nv("bcs_dist_solve");
    if (!d || !b_dev || !x_dev || (d->proc && !d->connected)) return BCS_ERR_ARG;
    if (!device_reachable(b_dev) || !device_reachable(x_dev)) return BCS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int held = (int)d->ranks.size();   // all ranks, or this process's one
    DistArgs D;
    memset(&D, 0, sizeof(D));
    D.params = d->dparams;
    D.nranks = held;
    D.rec_offset = d->proc ? d->rank * d->grid : 0;
    D.rec_total = d->total_ctas;
    D.bar_base = d->proc ? d->bar_base : 0u;
    D.sys = d->proc;
    D.cta0[0] = 0;
    for (int r = 0; r < held; ++r) {
        const bcs_dist_s::Rank& R = d->ranks[r];
        D.cta0[r + 1] = D.cta0[r] + R.ctas;
        KParams& P = d->hparams[r];
        memset(&P, 0, sizeof(P));
        P.n = R.nloc;
        P.ntiles = (R.nloc + 31) / 32;
        P.kind = d->kind;
        P.maxit = d->maxit;
        P.rr_m = d->opt.rr_m;
        P.rr_M = d->opt.rr_M;
        P.max_outer = d->opt.max_outer;
        P.mixed = d->vt_f32;
        P.hist_cap = d->opt.history_len;
        P.inner_maxit = d->opt.inner_maxit;
        P.inner_stall = d->opt.inner_stall;
        P.tol = d->tol;
        P.inner_tol = d->opt.inner_tol;
        P.spin_budget = spin_cycles(d->opt.spin_budget_ms);
        P.rowptr = R.rowptr;
        P.col = R.col;
        P.val64 = R.val64;
        P.val = d->vt_f32 ? (const void*)R.valin : (const void*)R.val64;
        P.x64 = R.x64 + R.nleft;
        P.b64 = b_dev + R.row0;
        for (int v = 0; v < NVEC; ++v) P.vec[v] = R.vecmem + ((size_t)v * (size_t)R.len + (size_t)R.nleft) * d->vbytes;
        P.partials = d->proc ? d->rec : d->partials;
        P.bar = d->bar;
        P.err = (int*)(d->bar + 4);
        P.hist = d->hist;
        P.scal = d->scal;
        P.out = d->out;
        P.row0 = R.row0;
        P.send_ptr = R.send_ptr;
        P.send_dst = R.send_dst;
        P.tile_send = R.tile_send;
        P.peer_vec = d->dpeer;
        P.bg = b_dev;
        P.xg = x_dev;
    }
    // process mode: the shared counter is not reset (every rank would race the
    // others' first arrivals); each rank adds the barriers it passed instead
    if (cudaMemcpyAsync(d->dparams, d->hparams, sizeof(KParams) * (size_t)held, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        (!d->proc && cudaMemsetAsync(d->bar, 0, 64, st) != cudaSuccess) ||
        cudaMemsetAsync(d->out, 0, sizeof(double) * NOUT, st) != cudaSuccess)
        return BCS_ERR_CUDA;
    cudaEventRecord(d->ev0, st);
    const int e = dist_dispatch(d, &D, d->grid, st, nullptr);
    cudaEventRecord(d->ev1, st);
    if (e != 0) return BCS_ERR_CUDA;
    int herr = 0;
    if (cudaMemcpyAsync(d->host_out, d->out, sizeof(double) * NOUT, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(d->host_out + NOUT, d->bar + 4, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return BCS_ERR_CUDA;
    memcpy(&herr, d->host_out + NOUT, sizeof(int));
    const double* o = d->host_out;
    const int status = herr ? herr : (int)o[O_STATUS];
    d->hist_len = (int)o[O_HISTLEN];
    if (d->proc) d->bar_base += (unsigned)o[O_SYNCS];
    if (res) {
        memset(res, 0, sizeof(*res));
        res->status = status;
        res->iterations = (int)o[O_ITERS];
        res->outer_steps = (int)o[O_OUTER];
        res->rr_steps = (int)o[O_RR];
        res->fallbacks = (int)o[O_FALLBACK];
        res->rel_res_recursive = o[O_RECREL];
        res->rel_res_true = o[O_TRUEREL];
        res->r0_norm = o[O_R0];
        res->grid_syncs = (int)o[O_SYNCS];
        res->reductions = (int)o[O_REDUCTIONS];
        res->spmv_passes = (int)o[O_SPMV];
        res->t_start = o[O_T0];
        res->t_end = o[O_T1];
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, d->ev0, d->ev1) == cudaSuccess) res->seconds = ms * 1e-3;
    }
    return status;
}

int bcs_dist_get_history(bcs_dist d, double* out, int cap, int* len) {
    if (!d || cap < 0) return BCS_ERR_ARG;
    const int avail = std::min(d->hist_len, d->opt.history_len);
    if (len) *len = avail;
    const int m = std::min(avail, cap);
    if (out && m > 0 && cudaMemcpy(out, d->hist, sizeof(double) * m, cudaMemcpyDeviceToHost) != cudaSuccess)
        return BCS_ERR_CUDA;
    return BCS_OK;
}

int bcs_dist_get_scalars(bcs_dist d, double* out, int cap, int* len) {
    if (!d || cap < 0) return BCS_ERR_ARG;
    const int avail = std::min(d->hist_len, d->opt.history_len);
    if (len) *len = avail;
    const int m = std::min(avail, cap);
    if (out && m > 0 && cudaMemcpy(out, d->scal, sizeof(double) * 4 * m, cudaMemcpyDeviceToHost) != cudaSuccess)
        return BCS_ERR_CUDA;
    return BCS_OK;
}

int bcs_dist_info(bcs_dist d, int rank, int64_t* row0, int64_t* nloc, int64_t* nleft, int64_t* nright,
                  int64_t* nsend, int* ctas) {
    if (!d || rank < 0 || rank >= d->nranks) return BCS_ERR_ARG;
    const int idx = d->proc ? (rank == d->rank ? 0 : -1) : rank;   // a process holds its own rank only
    if (idx < 0) return BCS_ERR_ARG;
    const bcs_dist_s::Rank& R = d->ranks[idx];
    if (row0) *row0 = R.row0;
    if (nloc) *nloc = R.nloc;
    if (nleft) *nleft = R.nleft;
    if (nright) *nright = R.nright;
    if (nsend) *nsend = R.nsend;
    if (ctas) *ctas = R.ctas;
    return BCS_OK;
}

}  // extern "C"
