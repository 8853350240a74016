// shard.cu -- one join split over several ranks (one process per GPU).
//
// Every rank builds the same grid index from the same points (the index
// build is deterministic up to the order of points inside a cell) and runs
// the search-and-refine kernel over its own contiguous range of work
// items.  A range starts and ends at the first work item of a cell, so a
// cell's query blocks all belong to one rank: the pairs a rank emits are
// exactly those whose home cell (the cell UNICOMP assigns the cell pair to)
// is one of them, and the ranks' outputs are disjoint and together the full
// result.  The only exchange is a sum of the ranks' counts, left to the
// caller (for example one all-reduce).
//
// Work items are (cell, block of 32 of its points), ordered by cell and
// block.  The ranges are balanced by estimated work: item k costs
//   c_k = K_k (q_k + 20) + 2000,
// with q_k its query points and K_k its candidate points (the points of the
// adjacent cells the search visits, found by the search's own range
// builder).  This follows the search kernel's time per item: a fixed part
// per item (building the candidate ranges), a part per candidate chunk
// (staging and unpacking the candidates, about twenty queries' worth of
// comparisons) and a part per candidate and query.  On skewed data a cell's
// cost grows with its population times its neighbours', so equal item
// counts would not be equal work.  The bound between ranks r - 1 and r is
// the cell start whose exclusive cost prefix is nearest to C r / w (C the
// total): of the two starts around the first item whose prefix reaches
// C r / w, the closer one (the later on a tie).  The bounds grow with r, so
// the ranges tile the items, and a rank's cost exceeds C / w by at most
// the cost of one cell.
#include <cstring>
#include <vector>

#include "join_dev.cuh"

namespace sj {

namespace {

constexpr int kCostWarps = 4;

__host__ __device__ inline uint64_t snap_to_cell_start(const uint32_t *item_block, uint64_t n,
                                                        uint64_t k) {
    while (k < n && item_block[k] != 0) ++k;
    return k;
}

// Estimated cost of every work item (see the file comment), one warp per
// item, and the sum of all costs.
template <int D, bool UNI>
__global__ void __launch_bounds__(kCostWarps * 32)
    item_cost_kernel(const JoinArgs a, const uint32_t *__restrict__ counts,
                     unsigned long long *__restrict__ cost, unsigned long long *total) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint2 *rt = reinterpret_cast<uint2 *>(smem + (size_t)warp * a.sm_ranges);
    const uint32_t ni = counts[1];
    const uint32_t n_cells = *a.ccells;
    unsigned long long acc = 0;
    for (uint32_t k = blockIdx.x * kCostWarps + warp; k < ni; k += gridDim.x * kCostWarps) {
        const uint2 it = a.items[k];
        const uint32_t h = it.x;
        const uint32_t cbeg = __ldg(&a.qG[h]), cend = __ldg(&a.qG[h + 1]);
        const uint32_t nq = min((uint32_t)kQueryBlock, cend - (cbeg + it.y * kQueryBlock));
        int32_t c[D];
        uint32_t odd = 0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            c[j] = __ldg(&a.qcc[(uint64_t)h * D + j]);
            odd |= ((uint32_t)c[j] & 1u) << j;
        }
        uint32_t nr, K;
        build_ranges<D, UNI>(c, odd, a, n_cells, lane, rt, nr, K);
        const unsigned long long v = (unsigned long long)K * (nq + 20) + 2000;
        if (lane == 0) cost[k] = v;
        acc += v;
        __syncwarp();
    }
    if (lane == 0 && acc) atomicAdd(total, acc);
}

// Costs scaled into 32 bits for the scan: c >> s with the shift s that
// keeps the total below 2^30, plus one (every item costs at least 1); zero
// for the unused entries up to cap, so that the scan's total is the items'.
__global__ void scale_cost_kernel(const unsigned long long *__restrict__ cost,
                                  const uint32_t *__restrict__ counts,
                                  const unsigned long long *__restrict__ total, uint64_t cap,
                                  uint32_t *__restrict__ c32) {
    const uint32_t ni = counts[1];
    const unsigned long long t = *total;
    const int bits = t ? 64 - __clzll((long long)t) : 0;
    const int sh = bits > 30 ? bits - 30 : 0;
    for (uint64_t k = blockIdx.x * blockDim.x + threadIdx.x; k < cap; k += (uint64_t)gridDim.x * blockDim.x)
        c32[k] = k < ni ? (uint32_t)(cost[k] >> sh) + 1u : 0u;
}

// One thread: the shard bounds of `rank` from the exclusive cost prefix
// (pre[k] = cost of the items before k, tot = all items).
__global__ void cost_bounds_kernel(const uint2 *__restrict__ items, const uint32_t *__restrict__ counts,
                                   const uint32_t *__restrict__ pre, const uint32_t *__restrict__ tot,
                                   int rank, int world, unsigned long long *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint64_t n = counts[1];
    const uint64_t T = *tot;
    for (int e = 0; e < 2; ++e) {
        const uint64_t target = T * (uint64_t)(rank + e) / (uint64_t)world;
        uint64_t lo = 0, hi = n;          // first k with pre[k] >= target (n if none)
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if ((uint64_t)pre[mid] < target) lo = mid + 1; else hi = mid;
        }
        uint64_t k = n;
        if (rank + e != world && n > 0) {
            if (lo < n && items[lo].y == 0) {
                k = lo;                       // the crossing item starts a cell
            } else {
                // the crossing item lies inside a cell (or is the last one):
                // the cell starts a < it < b around it, the nearer one
                const uint64_t last = lo < n ? lo : n - 1;
                const uint64_t a = last - items[last].y;
                uint64_t b = last + 1;
                while (b < n && items[b].y != 0) ++b;
                const uint64_t pb = b < n ? (uint64_t)pre[b] : T;
                k = (target - (uint64_t)pre[a] < pb - target) ? a : b;
            }
        }
        out[e] = k;
    }
}

typedef void (*CostFn)(const JoinArgs, const uint32_t *, unsigned long long *, unsigned long long *);

template <int D>
CostFn cost_fn(bool uni) { return uni ? item_cost_kernel<D, true> : item_cost_kernel<D, false>; }

CostFn pick_cost(int d, bool uni) {
    switch (d) {
        case 1: return cost_fn<1>(uni);
        case 2: return cost_fn<2>(uni);
        case 3: return cost_fn<3>(uni);
        case 4: return cost_fn<4>(uni);
        case 5: return cost_fn<5>(uni);
        case 6: return cost_fn<6>(uni);
        case 7: return cost_fn<7>(uni);
        case 8: return cost_fn<8>(uni);
        default: return nullptr;
    }
}

}  // namespace

sj_status shard_items(Error &err, const Index &ix, bool uni, int rank, int world, cudaStream_t s,
                      uint32_t *lo, uint32_t *hi) {
    JoinLaunch l;
    l.unicomp = uni ? 1 : 0;
    JoinArgs a;
    SJ_TRY(fill_join_args(err, ix, l, 0, 0xffffffffu, nullptr, 0, nullptr, nullptr, nullptr, 1, a));
    CostFn fn = pick_cost(a.d, uni);
    if (!fn) return fail(err, SJ_EINVAL, "unsupported dimension");
    const uint64_t cap = ix.g.n + 1;              // work items never exceed the points
    DevBuf cost, c32, tmp;
    auto run = [&]() -> sj_status {
        SJ_TRY(dev_alloc(err, cost, cap * 8, s));
        SJ_TRY(dev_alloc(err, c32, cap * 4, s));
        SJ_TRY(dev_alloc(err, tmp, 64, s));
        unsigned long long *t = static_cast<unsigned long long *>(tmp.p);
        uint32_t *tot32 = reinterpret_cast<uint32_t *>(t + 2);
        unsigned long long *out = t + 4;
        SJ_CUDA_TRY(cudaMemsetAsync(tmp.p, 0, 64, s));
        int dev = 0;
        SJ_CUDA_TRY(cudaGetDevice(&dev));
        const size_t smem = (size_t)a.sm_ranges * kCostWarps;
        SJ_CUDA_TRY(cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int blocks = 8 * sm_count(dev);
        const uint32_t *cnt = n_items_dev(ix) - 1;   // [0] |G|, [1] work items
        fn<<<blocks, kCostWarps * 32, smem, s>>>(a, cnt, static_cast<unsigned long long *>(cost.p), t);
        note_launch();
        SJ_CUDA_TRY(cudaGetLastError());
        scale_cost_kernel<<<blocks, 256, 0, s>>>(static_cast<const unsigned long long *>(cost.p), cnt, t,
                                                cap, static_cast<uint32_t *>(c32.p));
        note_launch();
        SJ_CUDA_TRY(cudaGetLastError());
        // the scan covers the item-array capacity (the count stays on the
        // device); the entries past the count are zero
        SJ_TRY(exclusive_scan_u32(err, static_cast<const uint32_t *>(c32.p), static_cast<uint32_t *>(c32.p),
                                  cap, tot32, s));
        cost_bounds_kernel<<<1, 32, 0, s>>>(static_cast<const uint2 *>(ix.items.p), cnt,
                                            static_cast<const uint32_t *>(c32.p), tot32, rank, world, out);
        note_launch();
        SJ_CUDA_TRY(cudaGetLastError());
        unsigned long long h[2] = {0, 0};
        SJ_CUDA_TRY(cudaMemcpyAsync(h, out, 16, cudaMemcpyDeviceToHost, s));
        SJ_CUDA_TRY(cudaStreamSynchronize(s));
        *lo = (uint32_t)h[0];
        *hi = (uint32_t)h[1];
        return SJ_OK;
    };
    const sj_status st = run();
    dev_free(cost, s);
    dev_free(c32, s);
    dev_free(tmp, s);
    return st;
}

}  // namespace sj

extern "C" SJ_API sj_status sj_shard_bounds(const uint32_t *item_block, uint64_t n_items, int rank,
                                            int world, uint64_t *lo, uint64_t *hi) {
    if ((!item_block && n_items) || !lo || !hi || world < 1 || rank < 0 || rank >= world)
        return SJ_EINVAL;
    *lo = sj::snap_to_cell_start(item_block, n_items, n_items * (uint64_t)rank / (uint64_t)world);
    *hi = sj::snap_to_cell_start(item_block, n_items, n_items * (uint64_t)(rank + 1) / (uint64_t)world);
    return SJ_OK;
}

extern "C" SJ_API sj_status sj_shard_bounds_cost(const uint32_t *item_block, const uint64_t *item_cost,
                                                 uint64_t n_items, int rank, int world, uint64_t *lo,
                                                 uint64_t *hi) {
    if (((!item_block || !item_cost) && n_items) || !lo || !hi || world < 1 || rank < 0 || rank >= world)
        return SJ_EINVAL;
    // exclusive cost prefix, pre[n] the total
    std::vector<unsigned __int128> pre(n_items + 1, 0);
    for (uint64_t k = 0; k < n_items; ++k) pre[k + 1] = pre[k] + item_cost[k];
    const uint64_t n = n_items;
    uint64_t b[2];
    for (int e = 0; e < 2; ++e) {
        b[e] = n;
        if (rank + e == world || n == 0) continue;
        const unsigned __int128 target = pre[n] * (unsigned)(rank + e) / (unsigned)world;
        uint64_t lo = 0;                  // first item whose prefix reaches the target
        while (lo < n && pre[lo] < target) ++lo;
        if (lo < n && item_block[lo] == 0) {
            b[e] = lo;
            continue;
        }
        const uint64_t last = lo < n ? lo : n - 1;
        const uint64_t a = last - item_block[last];
        uint64_t c = last + 1;
        while (c < n && item_block[c] != 0) ++c;
        b[e] = (target - pre[a] < pre[c] - target) ? a : c;
    }
    *lo = b[0];
    *hi = b[1];
    return SJ_OK;
}
