// fl_noalloc.cu -- nearest-open-facility assignment that allocates nothing.
//
// Some callers cannot let a library call cudaMalloc: applications that have
// reserved the whole device for their own memory pool (an allocation from
// elsewhere would fail or fragment it), and latency-critical loops for which
// an allocation's implicit device synchronisation is not acceptable.  For
// them this file offers the assignment step with its scratch memory (BFS
// values, level stamps, frontiers, counters) in one file-scope device array
// of fixed size.  The caller passes the graph, the open set and the outputs.
//
// Every GPU that loads the library holds the array until the process exits.
// All calls share it and it keeps the last call's contents: each call clears
// what must start at zero.  Calls that overlap on the GPU (from several
// streams or threads) race on the array and give undefined results.
#include <cstdio>
#include <mutex>

#include "fl_internal.cuh"

namespace fl {

// kernels of k_solve.cu / k_util.cu reused by this entry point
__global__ void k_snapshot(const int32_t* __restrict__ fr, const unsigned long long* __restrict__ n_fr,
                           const unsigned long long* __restrict__ X, unsigned long long* __restrict__ frval,
                           unsigned long long* __restrict__ reset_next, uint32_t* __restrict__ tstamp, uint32_t tval,
                           int32_t* __restrict__ touched, unsigned long long* __restrict__ n_touched);
__global__ void k_push(const int32_t* __restrict__ fr, const unsigned long long* __restrict__ frval,
                       const unsigned long long* __restrict__ n_fr, const int64_t* __restrict__ rowp,
                       const int32_t* __restrict__ cols, unsigned long long add, unsigned long long* __restrict__ X,
                       uint32_t* __restrict__ stamp, uint32_t sv, int32_t* __restrict__ fr_next,
                       unsigned long long* __restrict__ n_next);
__global__ void k_unpack_bfs(const unsigned long long* __restrict__ X, int64_t n, int32_t* __restrict__ label,
                             int32_t* __restrict__ dist);
__global__ void k_validate_csr(const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols, int64_t n,
                               int64_t nnz, Counters* ctr);

namespace {

constexpr int64_t kMaxN = 1 << 20;  // largest graph the fixed scratch serves
constexpr int kMaxDevices = 64;

// X (8 B) + snapshot values (8 B) + stamps (4 B) + two frontiers (4 B each) per
// vertex, then two frontier counters and a Counters block.
constexpr size_t kOffX = 0;
constexpr size_t kOffVal = kOffX + 8 * kMaxN;
constexpr size_t kOffStamp = kOffVal + 8 * kMaxN;
constexpr size_t kOffFr0 = kOffStamp + 4 * kMaxN;
constexpr size_t kOffFr1 = kOffFr0 + 4 * kMaxN;
constexpr size_t kOffCnt = kOffFr1 + 4 * kMaxN;
constexpr size_t kOffCtr = kOffCnt + 256;
constexpr size_t kScratchBytes = kOffCtr + 256;
static_assert(sizeof(Counters) <= 256, "the Counters block must fit its 256-byte slot of the scratch");
static_assert(2 * sizeof(unsigned long long) <= 256, "the frontier counters must fit their 256-byte slot");

static __device__ __align__(256) unsigned char noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
unsigned char* g_scratch_on[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
int scratch_address(unsigned char** out) {
    int dev = 0;
    FL_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) FL_FAIL(FL_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_on[dev]) {
        void* p = nullptr;
        FL_CUDA(cudaGetSymbolAddress(&p, noalloc_scratch));
        g_scratch_on[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_on[dev];
    return FL_OK;
}

// Sources: every open vertex starts at distance 0 with its own id as label.
__global__ void k_seed_open(const uint8_t* __restrict__ open, int64_t n, unsigned long long* __restrict__ X,
                            uint32_t* __restrict__ stamp, int32_t* __restrict__ fr,
                            unsigned long long* __restrict__ n_fr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t v = base + lane_id();
        const bool src = v < n && open[v] != 0;
        if (src) {
            X[v] = (unsigned long long)v;
            stamp[v] = 1u;
        }
        const long long at = warp_append(src, n_fr);
        if (at >= 0) fr[at] = (int32_t)v;
    }
}

int grid_for(int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace
}  // namespace fl

using namespace fl;

extern "C" int fl_assign_nearest_noalloc(int64_t n, const int64_t* row_off, const int32_t* cols, int64_t nnz,
                                         const uint8_t* open, int32_t* assign_out, int32_t* dist_out,
                                         void* stream) {
    if (n < 1 || n > kMaxN) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "n = %lld outside [1, %lld], the size of the fixed scratch", (long long)n,
                      (long long)kMaxN);
        FL_FAIL(FL_EINVAL, buf);
    }
    if (nnz < 0 || !row_off || (nnz > 0 && !cols) || !open || (!assign_out && !dist_out))
        FL_FAIL(FL_EINVAL, "bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* base = nullptr;
    FL_TRY(scratch_address(&base));
    unsigned long long* X = reinterpret_cast<unsigned long long*>(base + kOffX);
    unsigned long long* val = reinterpret_cast<unsigned long long*>(base + kOffVal);
    uint32_t* stamp = reinterpret_cast<uint32_t*>(base + kOffStamp);
    int32_t* fr[2] = {reinterpret_cast<int32_t*>(base + kOffFr0), reinterpret_cast<int32_t*>(base + kOffFr1)};
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + kOffCnt);
    Counters* ctr = reinterpret_cast<Counters*>(base + kOffCtr);

    // the CSR is checked on the device before any traversal
    FL_CUDA(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
    k_validate_csr<<<grid_for(n + nnz, 256), 256, 0, st>>>(row_off, cols, n, nnz, ctr);
    FL_CUDA(cudaGetLastError());
    unsigned long long err = 1;
    FL_CUDA(cudaMemcpyAsync(&err, &ctr->error, 8, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    if (err) FL_FAIL(FL_EINVAL, "invalid CSR (offsets must be monotone from 0 to nnz, ids in [0, n))");

    // scratch state of this call: values unset, stamps and counters zero
    FL_CUDA(cudaMemsetAsync(X, 0xff, (size_t)n * 8, st));
    FL_CUDA(cudaMemsetAsync(stamp, 0, (size_t)n * 4, st));
    FL_CUDA(cudaMemsetAsync(cnt, 0, 256, st));
    k_seed_open<<<grid_for(n, 256), 256, 0, st>>>(open, n, X, stamp, fr[0], &cnt[0]);
    FL_CUDA(cudaGetLastError());
    unsigned long long n_cur = 0;
    FL_CUDA(cudaMemcpyAsync(&n_cur, &cnt[0], 8, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    int cur = 0;
    uint32_t level = 0;
    while (n_cur > 0) {
        if ((int64_t)level > n) FL_FAIL(FL_ETIMEOUT, "BFS exceeded n levels");
        k_snapshot<<<grid_for((int64_t)n_cur, 256), 256, 0, st>>>(fr[cur], &cnt[cur], X, val, &cnt[cur ^ 1], nullptr,
                                                                  0, nullptr, nullptr);
        k_push<<<grid_for((int64_t)n_cur, 8), 256, 0, st>>>(fr[cur], val, &cnt[cur], row_off, cols, 1ULL << 32, X,
                                                            stamp, level + 2, fr[cur ^ 1], &cnt[cur ^ 1]);
        FL_CUDA(cudaGetLastError());
        FL_CUDA(cudaMemcpyAsync(&n_cur, &cnt[cur ^ 1], 8, cudaMemcpyDeviceToHost, st));
        FL_CUDA(cudaStreamSynchronize(st));
        cur ^= 1;
        ++level;
    }
    k_unpack_bfs<<<grid_for(n, 256), 256, 0, st>>>(X, n, assign_out, dist_out);
    FL_CUDA(cudaGetLastError());
    FL_CUDA(cudaStreamSynchronize(st));
    return FL_OK;
}
