// brute.cu -- the index-free comparator: every ordered pair (i, j) of the
// n points is tested with the exact FP64 predicate of Section III (each
// operation rounded on its own, no contraction).  O(n^2) evaluations; it
// exists to measure what the grid index and UNICOMP save (the paper's
// comparison of the indexed GPU join with a brute-force GPU join).
//
// Each block takes 128 query points (one per thread) and streams all points
// through shared memory in tiles of 256; a warp whose lanes find members for
// the same candidate reserves their output slots with one atomic and writes
// them with one store each.
#include <cmath>

#include "sj_internal.cuh"

namespace sj {

namespace {

constexpr int kBfThreads = 128;
constexpr int kBfTile = 256;

template <int D>
__global__ void __launch_bounds__(kBfThreads) brute_kernel(const double *__restrict__ pts, uint32_t n,
                                                           double E2, uint2 *__restrict__ out,
                                                           unsigned long long cap,
                                                           unsigned long long *__restrict__ counter) {
    __shared__ double tile[kBfTile * D];
    const uint32_t i = blockIdx.x * kBfThreads + threadIdx.x;
    const bool valid = i < n;
    double p[D];
#pragma unroll
    for (int j = 0; j < D; ++j) p[j] = valid ? pts[(size_t)i * D + j] : 0.0;
    const int lane = threadIdx.x & 31;
    for (uint32_t t0 = 0; t0 < n; t0 += kBfTile) {
        const uint32_t tn = min((uint32_t)kBfTile, n - t0);
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < tn * D; k += kBfThreads) tile[k] = pts[(size_t)t0 * D + k];
        __syncthreads();
        for (uint32_t c = 0; c < tn; ++c) {
            double s = 0.0;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const double t = __dsub_rn(p[j], tile[c * D + j]);
                s = __dadd_rn(s, __dmul_rn(t, t));
            }
            const bool hit = valid && s <= E2;
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (m) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(counter, (unsigned long long)__popc(m));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (hit) {
                    const unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
                    if (pos < cap) out[pos] = make_uint2(i, t0 + c);
                }
            }
        }
    }
}

typedef void (*BruteFn)(const double *, uint32_t, double, uint2 *, unsigned long long,
                        unsigned long long *);

BruteFn brute_fn(int d) {
    switch (d) {
        case 1: return brute_kernel<1>;
        case 2: return brute_kernel<2>;
        case 3: return brute_kernel<3>;
        case 4: return brute_kernel<4>;
        case 5: return brute_kernel<5>;
        case 6: return brute_kernel<6>;
        case 7: return brute_kernel<7>;
        case 8: return brute_kernel<8>;
        default: return nullptr;
    }
}

}  // namespace

sj_status brute_join(Error &err, const double *d_pts, uint64_t n, int d, double eps, uint2 *out,
                     uint64_t cap, unsigned long long *d_counter, cudaStream_t s) {
    BruteFn fn = brute_fn(d);
    if (!fn) return fail(err, SJ_EINVAL, "d must be in [1, 8]");
    const unsigned blocks = (unsigned)((n + kBfThreads - 1) / kBfThreads);
    fn<<<blocks, kBfThreads, 0, s>>>(d_pts, (uint32_t)n, eps * eps, out, cap, d_counter);
    note_launch();
    SJ_CUDA_TRY(cudaGetLastError());
    return SJ_OK;
}

}  // namespace sj
