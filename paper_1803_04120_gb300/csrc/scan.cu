// scan.cu -- device-wide exclusive prefix sum of uint32 values.
//
// Used by the index build to turn per-cell counts into the cell ranges of G
// and the dense lookup table, and per-cell work-item counts into item
// offsets.  Reduce-then-scan: each 4096-element tile is reduced, the tile
// sums are scanned (recursively), and every tile is scanned locally with its
// offset added.  Two passes over the data; the inputs here are at most a few
// tens of MB, so the scan is launch- rather than bandwidth-bound.
#include "sj_internal.cuh"

namespace sj {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread across the block; returns the
// thread's exclusive prefix and writes the block total to *total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0u;
        uint32_t wi = warp_incl_scan(w);
        if (lane < kScanThreads / 32) warp_sums[lane] = wi - w;
        if (lane == kScanThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    uint32_t r = warp_sums[warp] + incl - v;
    return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t *__restrict__ in,
                                                                   uint64_t n,
                                                                   uint32_t *__restrict__ sums) {
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint32_t v = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        uint64_t i = base + (uint64_t)k * kScanThreads + threadIdx.x;
        if (i < n) v += in[i];
    }
    __shared__ uint32_t total;
    (void)block_excl_scan(v, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Scans each tile: thread t owns elements base + t*kScanItems .. + kScanItems.
// Elements are staged through shared memory so the global loads and stores
// are coalesced.
__global__ void __launch_bounds__(kScanThreads) scan_tile_kernel(const uint32_t *in, uint32_t *out,
                                                                 uint64_t n,
                                                                 const uint32_t *__restrict__ offsets,
                                                                 uint32_t *d_total) {
    __shared__ uint32_t tile[kScanTile];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int li = k * kScanThreads + threadIdx.x;
        uint64_t i = base + li;
        tile[li] = i < n ? in[i] : 0u;
    }
    __syncthreads();
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = tile[threadIdx.x * kScanItems + k];
        s += v[k];
    }
    __shared__ uint32_t total;
    uint32_t pre = block_excl_scan(s, &total);
    uint32_t off = offsets ? offsets[blockIdx.x] : 0u;
    uint32_t run = off + pre;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        tile[threadIdx.x * kScanItems + k] = run;
        run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int li = k * kScanThreads + threadIdx.x;
        uint64_t i = base + li;
        if (i < n) out[i] = tile[li];
    }
    if (d_total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) *d_total = off + total;
}

}  // namespace

// Tile sums the scan below needs for n elements (two levels: up to 4096^2).
uint64_t scan_sums_needed(uint64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

// The same exclusive scan with its tile sums in a caller-provided device
// buffer (sums_cap entries) instead of freshly allocated memory.
sj_status exclusive_scan_u32_scratch(Error &err, const uint32_t *in, uint32_t *out, uint64_t n,
                                     uint32_t *d_total, uint32_t *sums, uint64_t sums_cap,
                                     cudaStream_t s) {
    if (n == 0) {
        if (d_total) SJ_CUDA_TRY(cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s));
        return SJ_OK;
    }
    const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        scan_tile_kernel<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, d_total); note_launch();
        SJ_CUDA_TRY(cudaGetLastError());
        return SJ_OK;
    }
    if (tiles > (uint64_t)kScanTile || tiles > sums_cap)
        return fail(err, SJ_ERANGE, "scan scratch too small");
    scan_reduce_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums); note_launch();
    scan_tile_kernel<<<1, kScanThreads, 0, s>>>(sums, sums, tiles, nullptr, d_total); note_launch();
    scan_tile_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums, nullptr); note_launch();
    SJ_CUDA_TRY(cudaGetLastError());
    return SJ_OK;
}

sj_status exclusive_scan_u32(Error &err, const uint32_t *in, uint32_t *out, uint64_t n,
                             uint32_t *d_total, cudaStream_t s) {
    if (n == 0) {
        if (d_total) SJ_CUDA_TRY(cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s));
        return SJ_OK;
    }
    const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles > 0x7fffffffULL) return fail(err, SJ_ERANGE, "scan too large");
    if (tiles == 1) {
        scan_tile_kernel<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, d_total); note_launch();
        SJ_CUDA_TRY(cudaGetLastError());
        return SJ_OK;
    }
    DevBuf sums;
    SJ_TRY(dev_alloc(err, sums, tiles * sizeof(uint32_t), s));
    uint32_t *ps = static_cast<uint32_t *>(sums.p);
    scan_reduce_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, ps); note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { dev_free(sums, s); set_cuda_error(err, e, "scan_reduce", __FILE__, __LINE__); return err.st; }
    sj_status st = exclusive_scan_u32(err, ps, ps, tiles, d_total, s);
    if (st != SJ_OK) { dev_free(sums, s); return st; }
    scan_tile_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, ps, nullptr); note_launch();
    e = cudaGetLastError();
    dev_free(sums, s);
    if (e != cudaSuccess) { set_cuda_error(err, e, "scan_tile", __FILE__, __LINE__); return err.st; }
    return SJ_OK;
}

}  // namespace sj
