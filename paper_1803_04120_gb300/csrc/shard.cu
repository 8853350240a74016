// shard.cu -- one join split over several ranks (one process per GPU).
//
// Every rank builds the same grid index from the same points (the index
// build is deterministic up to the order of points inside a cell) and runs
// the search-and-refine kernel over its own contiguous range of work
// items.  A range starts and ends at the first work item of a cell, so a
// cell's query blocks all belong to one rank: the pairs a rank emits are
// exactly those whose home cell (the cell UNICOMP assigns the cell pair to)
// is one of its cells, and the ranks' outputs are disjoint and together the
// full result.  The only exchange is a sum of the ranks' counts, left to the
// caller (for example one all-reduce).
//
// Work items are (cell, block of 32 of its points), ordered by cell and
// block, so the nominal split [n r / w, n (r + 1) / w) of the n items
// balances query blocks; each nominal bound moves forward to the next item
// whose block index is 0 (a cell start), or to n.
#include <cstring>

#include "sj_internal.cuh"

namespace sj {

namespace {

__host__ __device__ inline uint64_t snap_to_cell_start(const uint32_t *item_block, uint64_t n,
                                                        uint64_t k) {
    while (k < n && item_block[k] != 0) ++k;
    return k;
}

// One thread: the shard bounds of `rank` from the device work-item list.
__global__ void shard_bounds_kernel(const uint2 *__restrict__ items, const uint32_t *__restrict__ n_items,
                                    int rank, int world, unsigned long long *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint64_t n = *n_items;
    uint64_t b[2] = {n * (uint64_t)rank / (uint64_t)world, n * (uint64_t)(rank + 1) / (uint64_t)world};
    for (int e = 0; e < 2; ++e) {
        uint64_t k = b[e];
        while (k < n && items[k].y != 0) ++k;
        out[e] = k;
    }
}

}  // namespace

sj_status shard_items(Error &err, const Index &ix, int rank, int world, cudaStream_t s,
                      uint32_t *lo, uint32_t *hi) {
    DevBuf tmp;
    SJ_TRY(dev_alloc(err, tmp, 16, s));
    shard_bounds_kernel<<<1, 32, 0, s>>>(static_cast<const uint2 *>(ix.items.p), n_items_dev(ix), rank,
                                         world, static_cast<unsigned long long *>(tmp.p));
    note_launch();
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, tmp.p, 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(tmp, s);
    if (e != cudaSuccess) {
        set_cuda_error(err, e, "shard bounds", __FILE__, __LINE__);
        return err.st;
    }
    *lo = (uint32_t)h[0];
    *hi = (uint32_t)h[1];
    return SJ_OK;
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
