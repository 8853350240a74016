// noalloc.cu -- a self-join entry point that allocates no memory.
//
// Some callers cannot allocate device memory at all: code that runs inside
// another framework's memory budget with a pre-reserved pool, callers that
// must not call cudaMalloc while other work is being enqueued, or embedded
// use where every allocation has to be accounted for up front.  For them
// sj_selfjoin_noalloc runs the same index build and search-and-refine
// kernels as sj_selfjoin_device, but takes all its working memory from one
// fixed region declared below.  The caller passes the points and the pair
// buffer (both device memory); nothing else is allocated: no cudaMalloc,
// no cudaFree, no allocating library routine.
//
// The region is a file-scope __device__ array, so every GPU that loads the
// library holds it (kNoAllocBytes) until the process exits.  Host code may
// not use the array's name as a device address: the address is obtained with
// cudaGetSymbolAddress on the first call on each device (with that device
// current) and cached.  All calls share the region and it keeps the previous
// call's contents; the build clears what must start at zero.  Two calls
// whose work overlapped on the GPU would race on the region, so the library
// serialises them: a host mutex, held until the call's stream has finished.
// (Each process has its own copy of the region in its own CUDA context.)
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "sj_internal.cuh"

namespace {

constexpr uint64_t kNoAllocMaxPoints = 1ull << 16;     // 65,536 points
constexpr uint64_t kNoAllocMaxGridCells = 1ull << 20;  // dense lookup table entries
constexpr size_t kNoAllocBytes = (size_t)24 << 20;     // 24 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[64] = {nullptr};

sj_status say(char *msg, size_t msg_len, sj_status st, const char *text) {
    if (msg && msg_len) {
        std::snprintf(msg, msg_len, "%s", text);
    }
    return st;
}

bool on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" SJ_API sj_status sj_selfjoin_noalloc(const double *d_pts, uint64_t n, int d, double eps,
                                                uint32_t *d_pairs, uint64_t cap_pairs,
                                                uint64_t *count, void *stream, char *msg,
                                                size_t msg_len) {
    using namespace sj;
    if (msg && msg_len) msg[0] = '\0';
    if (!d_pts || !count || n == 0 || d < 1 || d > kMaxDim || !(eps > 0.0) || !std::isfinite(eps))
        return say(msg, msg_len, SJ_EINVAL, "invalid argument (d_pts, count, n > 0, d in [1,8], eps > 0 finite)");
    if (n > kNoAllocMaxPoints)
        return say(msg, msg_len, SJ_ERANGE, "n exceeds the 65536 points of the static scratch");
    if (cap_pairs && !d_pairs) return say(msg, msg_len, SJ_EINVAL, "d_pairs is NULL");
    if (!on_device(d_pts) || (cap_pairs && !on_device(d_pairs)))
        return say(msg, msg_len, SJ_EINVAL, "d_pts and d_pairs must be device memory");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return say(msg, msg_len, SJ_ECUDA, "no current CUDA device");
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return say(msg, msg_len, SJ_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
        }
        g_noalloc_addr[dev] = p;
    }
    unsigned char *region = static_cast<unsigned char *>(g_noalloc_addr[dev]);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // the last 256 bytes hold the join counters, cursor and error word
    const size_t misc_off = kNoAllocBytes - 256;
    unsigned long long *misc = reinterpret_cast<unsigned long long *>(region + misc_off);
    Error err;
    Index ix;
    sj_status st = build_index_static(err, d_pts, n, d, eps, region, misc_off, kNoAllocMaxGridCells,
                                      s, ix);
    if (st != SJ_OK) return say(msg, msg_len, st, err.msg.c_str());
    if (cudaMemsetAsync(misc, 0, 64, s) != cudaSuccess) {
        cudaGetLastError();
        return say(msg, msg_len, SJ_ECUDA, "cudaMemsetAsync failed");
    }
    JoinLaunch l;
    l.prec_fp32 = 1;
    l.unicomp = 1;
    l.grab = 1;
    st = launch_join(err, ix, l, 0, 0xffffffffu, reinterpret_cast<uint2 *>(d_pairs), cap_pairs,
                     misc, reinterpret_cast<uint32_t *>(misc + 4),
                     reinterpret_cast<uint32_t *>(misc + 5), 0, s, nullptr, nullptr);
    if (st != SJ_OK) return say(msg, msg_len, st, err.msg.c_str());
    unsigned long long h[8];
    if (cudaMemcpyAsync(h, misc, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        return say(msg, msg_len, SJ_ECUDA, cudaGetErrorString(e));
    }
    if ((uint32_t)h[5] & kErrTimeout)
        return say(msg, msg_len, SJ_ETIMEOUT, "a bounded device wait expired in the join kernel");
    *count = h[0];
    if (h[0] > cap_pairs) return say(msg, msg_len, SJ_EOVERFLOW, "output buffer too small for the pair count");
    return SJ_OK;
}
