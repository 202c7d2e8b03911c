// bcs_dot: the correctly rounded inner product on the device (the primitive
// behind the solver's a_i ... r_i), as a standalone entry point.
#include <string.h>

#include <algorithm>
#include <mutex>

#include "solver.cuh"

using namespace bcs;

namespace {

template <class VT>
__global__ void __launch_bounds__(kBlock) k_dot_partial(int64_t n, const VT* x, const VT* y, unsigned long long* recs) {
    __shared__ XStage<kWarps> s_x;
    WAcc a[10];
    wa_init10(a);
    const int lane = threadIdx.x & 31;
    for (int64_t b = blockIdx.x * (int64_t)kBlock + (threadIdx.x - lane); b < n; b += (int64_t)gridDim.x * kBlock) {
        const int64_t i = b + lane;
        const bool ok = i < n;
        wa_acc(a[0], ok ? x[i] : VT(0), ok ? y[i] : VT(0), ok);
    }
    flush_partials<1u>(a, s_x, recs + (size_t)blockIdx.x * NSLOT * kRec);
}

__global__ void __launch_bounds__(kBlock) k_dot_final(const unsigned long long* recs, int nblk, double* out) {
    __shared__ XStage<kWarps> s_x;
    __shared__ double s_out[10];
    reduce_partials<1>(recs, nblk, s_x, s_out);
    if (threadIdx.x == 0) *out = s_out[0];
}

}  // namespace

extern "C" int bcs_dot(int64_t n, const void* x, const void* y, int vec_f32, double* result, void* stream) {
    if (n < 0 || !result || (n > 0 && (!x || !y))) return BCS_ERR_ARG;
    if (n > 0 && (!device_reachable(x) || !device_reachable(y))) return BCS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((n + kBlock - 1) / kBlock, (int64_t)sms * 4));
    unsigned long long* recs = nullptr;
    double* dout = nullptr;
    int rc = BCS_OK;
    if (cudaMalloc(&recs, sizeof(unsigned long long) * (size_t)nblk * NSLOT * kRec) != cudaSuccess ||
        cudaMalloc(&dout, sizeof(double)) != cudaSuccess) {
        rc = BCS_ERR_OOM;
    } else {
        if (vec_f32) k_dot_partial<float><<<nblk, kBlock, 0, st>>>(n, (const float*)x, (const float*)y, recs);
        else k_dot_partial<double><<<nblk, kBlock, 0, st>>>(n, (const double*)x, (const double*)y, recs);
        k_dot_final<<<1, kBlock, 0, st>>>(recs, nblk, dout);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(result, dout, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = BCS_ERR_CUDA;
    }
    if (recs) cudaFree(recs);
    if (dout) cudaFree(dout);
    return rc;
}

// ---- bcs_dot_noalloc: the same inner product for callers that cannot allocate ----------
//
// The per-CTA partial records live in a file-scope device array instead of a
// cudaMalloc'd buffer: kNoAllocMaxCtas CTAs x one record of NSLOT x kRec
// words (256 x 512 B = 128 KiB), held by every GPU that loads the library
// until the process exits.  Host code cannot use the array's name as a device
// address, so its address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
namespace {

constexpr int kNoAllocMaxCtas = 256;
// each lane's 128-bit window holds at most 2^17 products: 256 CTAs x 256 lanes x 2^17
constexpr int64_t kNoAllocMaxN = (int64_t)kNoAllocMaxCtas * kBlock * (1 << 17);
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned long long g_noalloc_recs[(size_t)kNoAllocMaxCtas * NSLOT * kRec];

unsigned long long* g_noalloc_ptr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mu;

__global__ void __launch_bounds__(kBlock) k_dot_final1(const unsigned long long* recs, int nblk, double* out) {
    __shared__ XStage<kWarps> s_x;
    __shared__ double s_out[10];
    reduce_partials<1>(recs, nblk, s_x, s_out);
    if (threadIdx.x == 0) *out = s_out[0];
}

}  // namespace

extern "C" int bcs_dot_noalloc(int64_t n, const void* x, const void* y, int vec_f32, double* result_dev,
                               void* stream) {
    if (n < 0 || !result_dev || (n > 0 && (!x || !y))) return BCS_ERR_ARG;
    if (n > kNoAllocMaxN) return BCS_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BCS_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return BCS_ERR_ARG;
    unsigned long long* recs = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_recs) != cudaSuccess || !p) return BCS_ERR_CUDA;
            g_noalloc_ptr[dev] = (unsigned long long*)p;
        }
        recs = g_noalloc_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((n + kBlock - 1) / kBlock, kNoAllocMaxCtas));
    if (vec_f32) k_dot_partial<float><<<nblk, kBlock, 0, st>>>(n, (const float*)x, (const float*)y, recs);
    else k_dot_partial<double><<<nblk, kBlock, 0, st>>>(n, (const double*)x, (const double*)y, recs);
    k_dot_final1<<<1, kBlock, 0, st>>>(recs, nblk, result_dev);
    return cudaGetLastError() == cudaSuccess ? BCS_OK : BCS_ERR_CUDA;
}
