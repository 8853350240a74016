// sort.cu -- stable LSD radix sort of (uint64 key, uint32 value) pairs.
//
// The index build sorts points by linear cell id to form the lookup array A
// of Section IV-C when the grid is too large for the dense counting sort.
// Only the low `bits` bits of the keys are significant (the linear id is
// below the product of the cell counts), so the sort makes ceil(bits / 8)
// passes of 8 bits.  Each pass: per-tile digit histograms (digit-major), a
// device-wide exclusive scan of the histograms, and a stable scatter in
// which every warp ranks its items with __match_any_sync and the block
// combines the warps' digit counts.
#include "sj_internal.cuh"

namespace sj {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;                         // items per lane
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048
constexpr int kRadix = 256;

__global__ void __launch_bounds__(kSortThreads) sort_hist_kernel(const uint64_t *__restrict__ keys,
                                                                 uint64_t n, int shift,
                                                                 uint32_t ntiles,
                                                                 uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += kSortThreads) h[i] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        uint64_t i = base + (uint64_t)k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    for (int dgt = threadIdx.x; dgt < kRadix; dgt += kSortThreads)
        hist[(uint64_t)dgt * ntiles + blockIdx.x] = h[dgt];
}

// Warp w owns tile positions [w*256, (w+1)*256); item k of lane l sits at
// w*256 + k*32 + l, so (w, k, l) order is index order and ranking in that
// order keeps the sort stable.
__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(
    const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, uint64_t n, int shift,
    uint32_t ntiles, const uint32_t *__restrict__ offsets, uint64_t *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out) {
    __shared__ uint32_t wcount[kSortWarps][kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&wcount[0][0])[i] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kSortTile + (uint64_t)warp * (32 * kSortItems);
    uint64_t k_[kSortItems];
    uint32_t v_[kSortItems];
    uint32_t rank_[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        uint64_t i = base + (uint64_t)k * 32 + lane;
        bool valid = i < n;
        k_[k] = valid ? keys[i] : 0;
        v_[k] = valid ? vals[i] : 0;
        uint32_t dgt = valid ? (uint32_t)((k_[k] >> shift) & (kRadix - 1)) : (uint32_t)kRadix;
        unsigned peers = __match_any_sync(0xffffffffu, dgt);
        uint32_t before = 0;
        if (valid) before = wcount[warp][dgt];
        rank_[k] = before + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0) wcount[warp][dgt] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps for each digit
    for (int dgt = threadIdx.x; dgt < kRadix; dgt += kSortThreads) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            uint32_t c = wcount[w][dgt];
            wcount[w][dgt] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        uint64_t i = base + (uint64_t)k * 32 + lane;
        if (i < n) {
            uint32_t dgt = (uint32_t)((k_[k] >> shift) & (kRadix - 1));
            uint64_t pos = (uint64_t)offsets[(uint64_t)dgt * ntiles + blockIdx.x] +
                           wcount[warp][dgt] + rank_[k];
            keys_out[pos] = k_[k];
            vals_out[pos] = v_[k];
        }
    }
}

}  // namespace

sj_status radix_sort_pairs(Error &err, uint64_t *keys, uint32_t *vals, uint64_t n, int bits,
                           cudaStream_t s) {
    if (n <= 1 || bits <= 0) return SJ_OK;
    if (n >= (1ull << 32)) return fail(err, SJ_ERANGE, "sort: too many elements");
    const uint32_t ntiles = (uint32_t)((n + kSortTile - 1) / kSortTile);
    const int passes = (bits + 7) / 8;
    DevBuf kalt, valt, hist;
    SJ_TRY(dev_alloc(err, kalt, n * sizeof(uint64_t), s));
    sj_status st = dev_alloc(err, valt, n * sizeof(uint32_t), s);
    if (st == SJ_OK) st = dev_alloc(err, hist, (uint64_t)kRadix * ntiles * sizeof(uint32_t), s);
    if (st != SJ_OK) { dev_free(kalt, s); dev_free(valt, s); return st; }
    uint64_t *k_in = keys, *k_out = static_cast<uint64_t *>(kalt.p);
    uint32_t *v_in = vals, *v_out = static_cast<uint32_t *>(valt.p);
    uint32_t *ph = static_cast<uint32_t *>(hist.p);
    for (int p = 0; p < passes && st == SJ_OK; ++p) {
        const int shift = 8 * p;
        sort_hist_kernel<<<ntiles, kSortThreads, 0, s>>>(k_in, n, shift, ntiles, ph); note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { set_cuda_error(err, e, "sort_hist", __FILE__, __LINE__); st = err.st; break; }
        st = exclusive_scan_u32(err, ph, ph, (uint64_t)kRadix * ntiles, nullptr, s);
        if (st != SJ_OK) break;
        sort_scatter_kernel<<<ntiles, kSortThreads, 0, s>>>(k_in, v_in, n, shift, ntiles, ph, k_out,
                                                            v_out); note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) { set_cuda_error(err, e, "sort_scatter", __FILE__, __LINE__); st = err.st; break; }
        uint64_t *tk = k_in; k_in = k_out; k_out = tk;
        uint32_t *tv = v_in; v_in = v_out; v_out = tv;
    }
    if (st == SJ_OK && k_in != keys) {
        cudaError_t e = cudaMemcpyAsync(keys, k_in, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(vals, v_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) { set_cuda_error(err, e, "sort copy-back", __FILE__, __LINE__); st = err.st; }
    }
    dev_free(kalt, s);
    dev_free(valt, s);
    dev_free(hist, s);
    return st;
}

}  // namespace sj
