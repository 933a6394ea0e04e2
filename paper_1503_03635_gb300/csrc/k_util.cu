// k_util.cu -- errors, device buffers, scans, radix sort, CSR checks.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fl_internal.cuh"

namespace fl {

// ----------------------------------------------------------------- errors

static thread_local std::string t_err;
static thread_local int t_status = FL_OK;

void set_error(int status, const std::string& msg) {
    t_status = status;
    t_err = msg;
}

int status_of(cudaError_t e, const char* what, const char* file, int line) {
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    int st = (e == cudaErrorMemoryAllocation) ? FL_ENOMEM : FL_ECUDA;
    set_error(st, buf);
    return st;
}

int last_error(char* buf, size_t len) {
    if (buf && len) {
        size_t m = t_err.size() < len - 1 ? t_err.size() : len - 1;
        std::memcpy(buf, t_err.data(), m);
        buf[m] = 0;
    }
    return t_status;
}

// ----------------------------------------------------------------- profiling

static thread_local Prof* t_prof = nullptr;
static thread_local cudaStream_t t_stream = nullptr;

Prof* current_prof() { return t_prof; }
void set_current_prof(Prof* p, cudaStream_t st) {
    t_prof = p;
    t_stream = st;
}

int prof_begin(int cls) {
    Prof* p = t_prof;
    if (!p) return -1;
    p->launches[cls] += 1;
    if (!p->on) return -1;
    if (p->used * 2 + 2 > p->ev.size()) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            p->ev.push_back(e);
        }
    }
    size_t slot = p->used++;
    if (p->cls.size() < p->used) p->cls.resize(p->used);
    p->cls[slot] = cls;
    cudaEventRecord(p->ev[2 * slot], t_stream);
    return (int)slot;
}

void prof_end(int slot) {
    Prof* p = t_prof;
    if (!p || slot < 0) return;
    cudaEventRecord(p->ev[2 * slot + 1], t_stream);
}

int prof_drain(Prof* p) {
    if (!p || !p->used) return FL_OK;
    for (size_t i = 0; i < p->used; ++i) {
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, p->ev[2 * i], p->ev[2 * i + 1]);
        if (e != cudaSuccess) {
            p->used = 0;
            return status_of(e, "cudaEventElapsedTime", __FILE__, __LINE__);
        }
        p->ms[p->cls[i]] += ms;
    }
    p->used = 0;
    return FL_OK;
}

// ----------------------------------------------------------------- buffers
// Device buffers.  Buffers of destroyed handles (whose streams have been
// synchronised, so no work uses them any more) go to a per-device cache of
// idle blocks instead of cudaFree; dalloc takes the smallest cached block
// that fits (and is at most twice the request) before calling cudaMalloc.
// Repeated create/solve/destroy sequences then allocate nothing new and skip
// cudaMalloc/cudaFree, which are slow for the tens of GB a large graph holds.
// The cache holds at most half of the device's memory; a failed cudaMalloc
// releases it and retries.

namespace {

constexpr int kMaxPoolDevices = 64;

struct Pool {
    std::mutex mu;
    std::multimap<size_t, void*> blocks[kMaxPoolDevices];
    size_t bytes[kMaxPoolDevices] = {};
    size_t cap[kMaxPoolDevices] = {};
};

Pool& pool() {
    static Pool* p = new Pool();  // never destroyed: blocks live until the process exits
    return *p;
}

int current_device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxPoolDevices) return -1;
    return d;
}

void* pool_take(size_t bytes, size_t* got) {
    const int d = current_device();
    if (d < 0) return nullptr;
    Pool& P = pool();
    std::lock_guard<std::mutex> lock(P.mu);
    auto it = P.blocks[d].lower_bound(bytes);
    if (it == P.blocks[d].end() || it->first > 2 * bytes + (1 << 20)) return nullptr;
    void* p = it->second;
    *got = it->first;
    P.bytes[d] -= it->first;
    P.blocks[d].erase(it);
    return p;
}

void pool_release_all() {
    const int d = current_device();
    if (d < 0) return;
    Pool& P = pool();
    std::lock_guard<std::mutex> lock(P.mu);
    for (auto& kv : P.blocks[d]) cudaFree(kv.second);
    P.blocks[d].clear();
    P.bytes[d] = 0;
}

}  // namespace

int dalloc(DBuf& b, size_t bytes) {
    if (b.p && b.bytes >= bytes) return FL_OK;
    dfree(b);
    if (bytes == 0) bytes = 16;
    size_t got = 0;
    if (void* p = pool_take(bytes, &got)) {
        b.p = p;
        b.bytes = got;
        return FL_OK;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        pool_release_all();
        e = cudaMalloc(&b.p, bytes);
    }
    if (e != cudaSuccess) {
        b.p = nullptr;
        return status_of(e, "cudaMalloc", __FILE__, __LINE__);
    }
    b.bytes = bytes;
    return FL_OK;
}

int dgrow(DBuf& b, size_t bytes, size_t keep, cudaStream_t st) {
    if (b.p && b.bytes >= bytes) return FL_OK;
    DBuf nb;
    FL_TRY(dalloc(nb, bytes));
    cudaError_t e = cudaSuccess;
    if (b.p && keep) e = cudaMemcpyAsync(nb.p, b.p, keep, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        dfree(nb);
        return status_of(e, "dgrow copy", __FILE__, __LINE__);
    }
    dfree_idle(b);  // the stream is idle: nothing uses the old block any more
    b = nb;
    return FL_OK;
}

void dfree(DBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// For buffers no pending work uses (their handle's stream is synchronised).
void dfree_idle(DBuf& b) {
    if (!b.p) return;
    const int d = current_device();
    bool kept = false;
    if (d >= 0) {
        Pool& P = pool();
        std::lock_guard<std::mutex> lock(P.mu);
        if (P.cap[d] == 0) {
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) P.cap[d] = total_b / 2;
        }
        if (P.bytes[d] + b.bytes <= P.cap[d]) {
            P.blocks[d].insert({b.bytes, b.p});
            P.bytes[d] += b.bytes;
            kept = true;
        }
    }
    if (!kept) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

void dfree_after(cudaStream_t st, std::initializer_list<DBuf*> bufs) {
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        for (DBuf* b : bufs) dfree(*b);  // cudaFree waits for the device itself
        return;
    }
    for (DBuf* b : bufs) dfree_idle(*b);
}

// ----------------------------------------------------------------- scan
// Exclusive prefix sum with int64 output: tiles of 2048 items (256 threads x
// 8 consecutive items), reduce -> scan of tile sums (recursive) -> tile scan.

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ T block_excl_scan(T x, T* warp_tot, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = x;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        T y = __shfl_up_sync(kFull, incl, s);
        if (lane >= s) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            T y = __shfl_up_sync(kFull, wi, s);
            if (lane >= s) wi += y;
        }
        if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = wi - w;
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    T r = incl - x + warp_tot[warp];
    __syncthreads();
    return r;
}

template <class Tin>
__global__ void k_tile_sums(const Tin* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
    __shared__ int64_t wt[32];
    __shared__ int64_t tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += (int64_t)in[base + i];
    block_excl_scan<int64_t>(s, wt, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <class Tin>
__global__ void k_tile_scan(const Tin* __restrict__ in, int64_t n, const int64_t* __restrict__ offs,
                            int64_t* __restrict__ out) {
    __shared__ int64_t wt[32];
    __shared__ int64_t tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? (int64_t)in[base + i] : 0;
        s += v[i];
    }
    int64_t run = block_excl_scan<int64_t>(s, wt, &tot) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

static size_t scan_tmp_bytes(int64_t n) {
    size_t b = 0;
    while (n > kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        b += 2 * (size_t)n * sizeof(int64_t) + 256;
    }
    return b + 256;
}

template <class Tin>
static int scan_rec(const Tin* in, int64_t* out, int64_t n, cudaStream_t st, char* tmp, int cls) {
    if (n <= 0) return FL_OK;
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        FL_LAUNCH(cls, k_tile_scan<Tin><<<1, kScanThreads, 0, st>>>(in, n, nullptr, out));
        FL_CUDA(cudaGetLastError());
        return FL_OK;
    }
    int64_t* sums = reinterpret_cast<int64_t*>(tmp);
    int64_t* offs = sums + tiles;
    char* next = reinterpret_cast<char*>(offs + tiles);
    next += (256 - (reinterpret_cast<uintptr_t>(next) & 255)) & 255;
    FL_LAUNCH(cls, k_tile_sums<Tin><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, sums));
    FL_CUDA(cudaGetLastError());
    FL_TRY(scan_rec<int64_t>(sums, offs, tiles, st, next, cls));
    FL_LAUNCH(cls, k_tile_scan<Tin><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, offs, out));
    FL_CUDA(cudaGetLastError());
    return FL_OK;
}

int scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st, DBuf& tmp, int cls) {
    FL_TRY(dalloc(tmp, scan_tmp_bytes(n)));
    return scan_rec<int64_t>(in, out, n, st, tmp.as<char>(), cls);
}

int scan_exclusive_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t st, DBuf& tmp,
                              int cls) {
    FL_TRY(dalloc(tmp, scan_tmp_bytes(n)));
    return scan_rec<int32_t>(in, out, n, st, tmp.as<char>(), cls);
}

// ----------------------------------------------------------------- radix sort
// Stable LSD radix sort of (hi, lo) 128-bit keys with a uint32 payload,
// 4-bit digits (32 passes, lo word first).  Per pass: per-tile digit
// histogram -> exclusive scan in digit-major order -> stable scatter, where
// each thread owns 8 consecutive items and per-digit offsets come from a
// block scan of 16 packed 16-bit counters (4 x uint64 words).

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void k_digit_hist(const uint64_t* __restrict__ key, int64_t n, int shift, int nblocks,
                             int32_t* __restrict__ hist) {
    __shared__ int32_t h[16];
    if (threadIdx.x < 16) h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)threadIdx.x * kSortItems;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i)
        if (base + i < n) atomicAdd(&h[(key[base + i] >> shift) & 15], 1);
    __syncthreads();
    if (threadIdx.x < 16) hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_digit_scatter(const uint64_t* __restrict__ key, const uint64_t* __restrict__ hi_in,
                                const uint64_t* __restrict__ lo_in, const uint32_t* __restrict__ val_in,
                                int64_t n, int shift, int nblocks, const int64_t* __restrict__ offs,
                                uint64_t* __restrict__ hi_out, uint64_t* __restrict__ lo_out,
                                uint32_t* __restrict__ val_out) {
    __shared__ uint64_t wt[4][32];
    __shared__ uint64_t tot[4];
    int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)threadIdx.x * kSortItems;
    int dig[kSortItems];
    uint64_t cnt[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        dig[i] = (base + i < n) ? (int)((key[base + i] >> shift) & 15) : -1;
        if (dig[i] >= 0) cnt[dig[i] >> 2] += 1ULL << (16 * (dig[i] & 3));
    }
    uint64_t ex[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) ex[w] = block_excl_scan<uint64_t>(cnt[w], wt[w], &tot[w]);
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        int d = dig[i];
        if (d < 0) continue;
        int w = d >> 2, sh = 16 * (d & 3);
        int64_t local = (int64_t)((ex[w] >> sh) & 0xffff);
        ex[w] += 1ULL << sh;
        int64_t pos = offs[(int64_t)d * nblocks + blockIdx.x] + local;
        hi_out[pos] = hi_in[base + i];
        lo_out[pos] = lo_in[base + i];
        val_out[pos] = val_in[base + i];
    }
}

int sort_pairs_u128(uint64_t* hi, uint64_t* lo, uint32_t* val, int64_t n, cudaStream_t st, DBuf& tmp, int cls,
                    int pass_begin, int pass_end) {
    if (pass_begin < 0 || pass_end > 32 || pass_begin > pass_end || ((pass_end - pass_begin) & 1))
        FL_FAIL(FL_EINVAL, "radix sort: bad pass range");
    uint32_t digits = 0;
    for (int p = pass_begin; p < pass_end; ++p) digits |= 1u << p;
    return sort_pairs_u128_digits(hi, lo, val, n, st, tmp, cls, digits);
}

int sort_pairs_u128_digits(uint64_t* hi, uint64_t* lo, uint32_t* val, int64_t n, cudaStream_t st, DBuf& tmp,
                           int cls, uint32_t digits) {
    if (n <= 1 || digits == 0) return FL_OK;
    int nblocks = (int)((n + kSortTile - 1) / kSortTile);
    int64_t hn = 16LL * nblocks;
    size_t need = (size_t)n * (8 + 8 + 4) + 256 * 8 + (size_t)hn * (4 + 8) + scan_tmp_bytes(hn);
    FL_TRY(dalloc(tmp, need));
    char* p = tmp.as<char>();
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~size_t(255);
        return r;
    };
    uint64_t* hi2 = reinterpret_cast<uint64_t*>(take((size_t)n * 8));
    uint64_t* lo2 = reinterpret_cast<uint64_t*>(take((size_t)n * 8));
    uint32_t* val2 = reinterpret_cast<uint32_t*>(take((size_t)n * 4));
    int32_t* hist = reinterpret_cast<int32_t*>(take((size_t)hn * 4));
    int64_t* offs = reinterpret_cast<int64_t*>(take((size_t)hn * 8));
    char* stmp = take(scan_tmp_bytes(hn));
    uint64_t *ahi = hi, *alo = lo, *bhi = hi2, *blo = lo2;
    uint32_t *aval = val, *bval = val2;
    for (int pass = 0; pass < 32; ++pass) {
        if (!((digits >> pass) & 1u)) continue;
        const uint64_t* key = pass < 16 ? alo : ahi;
        int shift = 4 * (pass & 15);
        FL_LAUNCH(cls, k_digit_hist<<<nblocks, kSortThreads, 0, st>>>(key, n, shift, nblocks, hist));
        FL_CUDA(cudaGetLastError());
        FL_TRY(scan_rec<int32_t>(hist, offs, hn, st, stmp, cls));
        FL_LAUNCH(cls, k_digit_scatter<<<nblocks, kSortThreads, 0, st>>>(key, ahi, alo, aval, n, shift, nblocks, offs,
                                                          bhi, blo, bval));
        FL_CUDA(cudaGetLastError());
        std::swap(ahi, bhi);
        std::swap(alo, blo);
        std::swap(aval, bval);
    }
    if (__builtin_popcount(digits) & 1) {  // an odd number of passes: copy the result back
        FL_CUDA(cudaMemcpyAsync(hi, ahi, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
        FL_CUDA(cudaMemcpyAsync(lo, alo, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
        FL_CUDA(cudaMemcpyAsync(val, aval, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    }
    return FL_OK;
}

// ----------------------------------------------------------------- CSR checks

__global__ void k_validate_csr(const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                               int64_t n, int64_t nnz, Counters* ctr) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (rowp[i] > rowp[i + 1] || rowp[i] < 0) atomicOr(&ctr->error, 1ULL);
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        int32_t c = cols[e];
        if (c < 0 || c >= n) atomicOr(&ctr->error, 2ULL);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rowp[0] != 0 || rowp[n] != nnz) atomicOr(&ctr->error, 4ULL);
    }
}

int read_counters(fl_graph* g) {
    FL_CUDA(cudaMemcpyAsync(g->h_ctr, g->ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, g->stream));
    FL_CUDA(cudaStreamSynchronize(g->stream));
    return FL_OK;
}

int validate_csr(fl_graph* g) {
    FL_CUDA(cudaMemsetAsync(g->ctr.p, 0, sizeof(Counters), g->stream));
    FL_LAUNCH(kProfOther, k_validate_csr<<<152 * 8, 256, 0, g->stream>>>(g->rowp.as<int64_t>(), g->cols.as<int32_t>(), g->n,
                                                    g->nnz, g->ctr.as<Counters>()));
    FL_CUDA(cudaGetLastError());
    FL_TRY(read_counters(g));
    if (g->h_ctr->error) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "invalid CSR (flags 0x%llx: 1=offsets decrease, 2=id out of range, "
                      "4=row_off[0]!=0 or row_off[n]!=nnz)", (unsigned long long)g->h_ctr->error);
        FL_FAIL(FL_EINVAL, buf);
    }
    return FL_OK;
}

}  // namespace fl
