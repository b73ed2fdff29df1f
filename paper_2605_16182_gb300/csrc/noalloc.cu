// noalloc.cu -- an entry point that never allocates device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a fixed memory
// plan (a host framework that owns all device memory through its own pool
// and forbids foreign allocations), or a latency-critical loop that must not
// pay cudaMalloc's implicit device synchronisation after start-up.  For them,
// tempest_sort_batch_noalloc sorts one edge batch by timestamp (the batch
// sort every ingest starts with) using scratch that lives in this file's
// static device array instead of memory requested at run time.
//
// The array is part of the library image: every GPU that loads the library
// holds TEMPEST_NOALLOC_SCRATCH_BYTES of it until the process exits.  All
// calls share it, and it keeps whatever the last call left there; nothing in
// it has to start at zero, because every sort pass writes the histogram and
// the key / value buffers it later reads.  Calls whose work overlaps on the
// GPU (different streams, or different host threads) race on the array.
#include <cuda.h>

#include <mutex>

#include "engine.cuh"
#include "prims.cuh"
#include "sortscan.cuh"

namespace tw {

namespace {

constexpr int64_t NOALLOC_MAX_EDGES = TEMPEST_NOALLOC_MAX_EDGES;
constexpr int64_t NOALLOC_MAX_BLOCKS = (NOALLOC_MAX_EDGES + SORT_TILE - 1) / SORT_TILE;

// layout of the scratch array (byte offsets, each 256-byte aligned)
constexpr size_t OFF_K0 = 0;
constexpr size_t OFF_K1 = OFF_K0 + sizeof(unsigned long long) * NOALLOC_MAX_EDGES;
constexpr size_t OFF_V0 = OFF_K1 + sizeof(unsigned long long) * NOALLOC_MAX_EDGES;
constexpr size_t OFF_V1 = OFF_V0 + sizeof(uint32_t) * NOALLOC_MAX_EDGES;
constexpr size_t OFF_HIST = OFF_V1 + sizeof(uint32_t) * NOALLOC_MAX_EDGES;
constexpr size_t SCRATCH_BYTES = OFF_HIST + sizeof(uint32_t) * (RADIX * NOALLOC_MAX_BLOCKS + 64);
static_assert(SCRATCH_BYTES <= TEMPEST_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the declared size");
static_assert(OFF_K1 % 256 == 0 && OFF_V0 % 256 == 0 && OFF_V1 % 256 == 0 && OFF_HIST % 256 == 0,
              "scratch sections must stay 256-byte aligned");

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[TEMPEST_NOALLOC_SCRATCH_BYTES];

// Signed timestamps as unsigned keys with the same order.
struct SignedTsLoader {
    const int64_t *ts;
    __device__ __forceinline__ unsigned long long key(int64_t i) const
    {
        return (unsigned long long)ts[i] ^ 0x8000000000000000ull;
    }
    __device__ __forceinline__ uint32_t val(int64_t i) const { return (uint32_t)i; }
};

__global__ void k_noalloc_gather(const uint32_t *__restrict__ perm, const int32_t *__restrict__ src,
                                 const int32_t *__restrict__ dst, const int64_t *__restrict__ ts, int64_t n,
                                 int32_t *osrc, int32_t *odst, int64_t *ots)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = perm[i];
        osrc[i] = src[p];
        odst[i] = dst[p];
        ots[i] = ts[p];
    }
}

// Device address of the scratch array, looked up once per device and
// context with that device current (a host-side use of the symbol's name
// would not be a device address).  The address belongs to the context that
// loaded the module: after cudaDeviceReset the next context may load it
// elsewhere, so each cached address carries its context's unique id and is
// looked up again when the current context's id differs.
struct ScratchAddr {
    unsigned long long ctx_id;
    unsigned char *p;
};
static ScratchAddr g_scratch_addr[64];
static std::mutex g_scratch_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (0 when there is none or
// the driver does not report one).
static unsigned long long current_ctx_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess && qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrentFn>(a);
            get_id = reinterpret_cast<CtxGetIdFn>(b);
        }
        cudaGetLastError();
        resolved = true;
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

static int scratch_for_current_device(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, TEMPEST_ECUDA, "tempest_sort_batch_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= 64) return fail(nullptr, TEMPEST_EINVAL, "tempest_sort_batch_noalloc: device %d", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const unsigned long long id = current_ctx_id();
    ScratchAddr &c = g_scratch_addr[dev];
    if (!c.p || id == 0 || c.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            c.p = nullptr;
            return fail(nullptr, TEMPEST_ECUDA, "tempest_sort_batch_noalloc: cudaGetSymbolAddress: %s",
                        cudaGetErrorString(e));
        }
        c.p = static_cast<unsigned char *>(p);
        c.ctx_id = current_ctx_id();  // the lookup made the device's primary context current
    }
    *out = c.p;
    return TEMPEST_OK;
}

}  // namespace tw

using namespace tw;

extern "C" int tempest_sort_batch_noalloc(const int32_t *src, const int32_t *dst, const int64_t *ts, int64_t n,
                                          int32_t *out_src, int32_t *out_dst, int64_t *out_ts, void *stream)
{
    if (n < 0) return fail(nullptr, TEMPEST_EINVAL, "tempest_sort_batch_noalloc: n = %lld < 0", (long long)n);
    if (n > NOALLOC_MAX_EDGES)
        return fail(nullptr, TEMPEST_EINVAL,
                    "tempest_sort_batch_noalloc: n = %lld exceeds the maximum of %lld edges (fixed scratch)",
                    (long long)n, (long long)NOALLOC_MAX_EDGES);
    if (n == 0) return TEMPEST_OK;
    const void *ptrs[6] = {src, dst, ts, out_src, out_dst, out_ts};
    for (const void *p : ptrs)
        if (!is_device_ptr(p))
            return fail(nullptr, TEMPEST_EINVAL, "tempest_sort_batch_noalloc: every array must be device memory");
    unsigned char *base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long *kb[2] = {reinterpret_cast<unsigned long long *>(base + OFF_K0),
                                 reinterpret_cast<unsigned long long *>(base + OFF_K1)};
    uint32_t *vb[2] = {reinterpret_cast<uint32_t *>(base + OFF_V0), reinterpret_cast<uint32_t *>(base + OFF_V1)};
    uint32_t *hist = reinterpret_cast<uint32_t *>(base + OFF_HIST);
    // all 64 key bits: no host read-back of the timestamp range is needed
    SignedTsLoader ld{ts};
    const int r = radix_sort_launch<unsigned long long>(ld, n, 64, kb, vb, hist, st, nullptr);
    int64_t grid = (n + 255) / 256;
    if (grid > 1024) grid = 1024;
    k_noalloc_gather<<<(unsigned)grid, 256, 0, st>>>(vb[r], src, dst, ts, n, out_src, out_dst, out_ts);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(nullptr, TEMPEST_ECUDA, "tempest_sort_batch_noalloc: launch: %s", cudaGetErrorString(e));
    return TEMPEST_OK;
}
