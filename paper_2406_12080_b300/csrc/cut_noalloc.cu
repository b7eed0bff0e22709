// Cut selection without any device allocation (h3dgs_select_cut_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs inside another framework's allocator-managed
// region or memory budget, real-time loops that must not hit the driver's allocator (it can
// synchronise the device), and hosts whose memory is fully partitioned up front.  For them this
// entry point computes the cut of one camera into buffers the caller already owns, with its
// scratch (selection bits, per-block counts, the total) in a fixed file-scope device array instead
// of context workspace.  It needs no context and no upload: it reads the caller's box and topology
// arrays directly.
//
// The scratch array is shared by every call in the process on a given device and keeps the last
// call's contents; each call writes every scratch word it later reads before reading it.  Calls
// whose kernels overlap on the GPU (different streams, or different host threads) race on it.
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace h3dgs {

namespace {

constexpr int64_t NA_MAX_NODES = H3DGS_NOALLOC_MAX_NODES;   // 2^24
constexpr int NA_MASK_WORDS = (int)(NA_MAX_NODES / 32);     // one bit per node
constexpr int NA_MAX_BLOCKS = 4096;                         // per-block counts of the scan
constexpr int NA_BLOCK = 256;
constexpr int NA_WORDS = NA_MASK_WORDS + NA_MAX_BLOCKS + 4; // + total (2 words) + padding

// Scratch of the no-allocation cut: [mask words | block counts | total lo, hi | pad], 2.02 MB.
static __device__ __align__(256) uint32_t g_noalloc_scratch[NA_WORDS];

// Derived camera values in the same fixed fp32 order as the context path's set-up kernel.
__device__ __forceinline__ DevCam na_camera(const h3dgs_camera& c) {
    DevCam d;
    camera_centre(c, d.c);
    d.f = fmaxf(c.fx, c.fy);
    d.tau = c.tau;
    return d;
}

__device__ __forceinline__ bool na_test(const DevCam& cam, const h3dgs_hierarchy& h, int64_t v, float* en, float* ep) {
    const float* lo = h.box_min + 3 * v;
    const float* hi = h.box_max + 3 * v;
    *en = granularity(cam, lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]);
    const bool leaf = h.child_count[v] == 0;
    const int32_t p = h.parent[v];
    *ep = __int_as_float(0x7f800000);
    bool parent_ok = true;
    if (p >= 0) {
        const float* plo = h.box_min + 3 * (int64_t)p;
        const float* phi = h.box_max + 3 * (int64_t)p;
        *ep = granularity(cam, plo[0], plo[1], plo[2], phi[0], phi[1], phi[2]);
        parent_ok = *ep >= cam.tau;
    }
    return ((*en < cam.tau) || leaf) && parent_ok;
}

__global__ void __launch_bounds__(NA_BLOCK) na_mark_kernel(h3dgs_hierarchy h, h3dgs_camera c, int64_t chunk,
                                                           uint32_t* __restrict__ scratch) {
    __shared__ uint32_t s_count;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    const DevCam cam = na_camera(c);
    const int lane = threadIdx.x & 31;
    const int64_t base = blockIdx.x * chunk;
    const int64_t end = min(base + chunk, h.n_nodes);
    for (int64_t v0 = base; v0 < end; v0 += NA_BLOCK) {
        const int64_t v = v0 + threadIdx.x;
        float en, ep;
        const bool sel = v < end && na_test(cam, h, v, &en, &ep);
        const uint32_t word = __ballot_sync(0xffffffffu, sel);
        if (lane == 0 && v < end) {
            scratch[v >> 5] = word;
            if (word) atomicAdd(&s_count, (uint32_t)__popc(word));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) scratch[NA_MASK_WORDS + blockIdx.x] = s_count;
}

// exclusive scan of the G block counts in place; total to the two total words and to the offsets
__global__ void __launch_bounds__(1024) na_scan_kernel(int G, int64_t capacity, uint32_t* __restrict__ scratch,
                                                       int64_t* __restrict__ cut_offsets) {
    __shared__ uint32_t s[1024];
    uint32_t* cnt = scratch + NA_MASK_WORDS;
    const int per = (G + 1023) / 1024;
    const int i0 = threadIdx.x * per, i1 = min(G, i0 + per);
    uint32_t sum = 0;
    for (int i = i0; i < i1; ++i) sum += cnt[i];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t x = (int)threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += x;
        __syncthreads();
    }
    uint32_t run = s[threadIdx.x] - sum;
    for (int i = i0; i < i1; ++i) { const uint32_t x = cnt[i]; cnt[i] = run; run += x; }
    if (threadIdx.x == 1023) {
        const int64_t total = s[1023];
        scratch[NA_MASK_WORDS + NA_MAX_BLOCKS] = (uint32_t)(total & 0xffffffffu);
        scratch[NA_MASK_WORDS + NA_MAX_BLOCKS + 1] = (uint32_t)(total >> 32);
        cut_offsets[0] = 0;
        cut_offsets[1] = total < capacity ? total : capacity;
    }
}

__global__ void __launch_bounds__(NA_BLOCK) na_write_kernel(h3dgs_hierarchy h, h3dgs_camera c, int64_t chunk,
                                                            const uint32_t* __restrict__ scratch, int64_t capacity,
                                                            int32_t* __restrict__ cut_ids, float* __restrict__ cut_t) {
    __shared__ uint32_t s_warp[NA_BLOCK / 32];
    __shared__ int64_t s_run;
    const DevCam cam = na_camera(c);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = blockIdx.x * chunk;
    const int64_t end = min(base + chunk, h.n_nodes);
    if (threadIdx.x == 0) s_run = scratch[NA_MASK_WORDS + blockIdx.x];
    __syncthreads();
    for (int64_t v0 = base; v0 < end; v0 += NA_BLOCK) {
        const int64_t v = v0 + threadIdx.x;
        const uint32_t word = (v0 + warp * 32 < end) ? scratch[(v0 >> 5) + warp] : 0u;
        const bool sel = (word >> lane) & 1u;
        if (lane == 0) s_warp[warp] = __popc(word);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int i = 0; i < NA_BLOCK / 32; ++i) {
            before += (i < warp) ? s_warp[i] : 0u;
            total += s_warp[i];
        }
        const int64_t pos = s_run + before + __popc(word & ((1u << lane) - 1u));
        if (sel && pos < capacity) {
            cut_ids[pos] = (int32_t)v;
            if (cut_t) {
                float en, ep;
                na_test(cam, h, v, &en, &ep);
                cut_t[pos] = h.parent[v] >= 0 ? parent_weight(cam.tau, en, ep) : 0.0f;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_run += total;
        __syncthreads();
    }
}

// Device address of the scratch array, looked up once per device and context: the address belongs
// to the module loaded into the device's current context, so a new context (after a device reset,
// or the primary context torn down and created again) needs a new look-up.
constexpr int NA_MAX_DEVICES = 64;
struct ScratchAddr {
    void* ctx;
    uint32_t* ptr;
};
ScratchAddr g_scratch[NA_MAX_DEVICES] = {};
std::mutex g_scratch_mutex;

// The driver's cuCtxGetCurrent, reached through the runtime (the library does not link libcuda).
typedef int (*CtxGetCurrentFn)(void**);
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(f);
    }();
    return fn;
}

void* current_context() {
    void* c = nullptr;
    CtxGetCurrentFn fn = ctx_get_current();
    if (!fn || fn(&c) != 0) return nullptr;
    return c;
}

template <typename... KArgs, typename... Args>
cudaError_t na_launch(void (*kernel)(KArgs...), int grid, int block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace

}  // namespace h3dgs

using namespace h3dgs;

extern "C" h3dgs_status h3dgs_select_cut_noalloc(const h3dgs_hierarchy* hier, const h3dgs_camera* cam,
                                                 int32_t* cut_ids, float* cut_t, int64_t* cut_offsets,
                                                 int64_t capacity, int64_t* total_out, void* cuda_stream) {
    if (!hier || !cam || !cut_offsets || capacity < 0 || (capacity > 0 && !cut_ids)) return H3DGS_ERR_INVALID_ARG;
    if (!hier->box_min || !hier->box_max || !hier->parent || !hier->child_count || hier->n_nodes < 1)
        return H3DGS_ERR_INVALID_ARG;
    if (hier->n_nodes > NA_MAX_NODES) return H3DGS_ERR_CAPACITY;  // beyond the fixed scratch
    if (!(cam->fx > 0) || !(cam->fy > 0) || !(cam->tau >= 0)) return H3DGS_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return H3DGS_ERR_NO_DEVICE;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return H3DGS_ERR_INVALID_ARG;
    uint32_t* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        void* ctx = current_context();
        if (!g_scratch[dev].ptr || !ctx || ctx != g_scratch[dev].ctx) {
            // first call on this device and context (which are current): resolve the array's device
            // address (this also creates the primary context if none is current yet)
            uint32_t* p = nullptr;
            if (cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch) != cudaSuccess || !p)
                return H3DGS_ERR_CUDA;
            g_scratch[dev].ptr = p;
            g_scratch[dev].ctx = current_context();
        }
        scratch = g_scratch[dev].ptr;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    const int64_t N = hier->n_nodes;
    int64_t chunk = ((N + NA_MAX_BLOCKS - 1) / NA_MAX_BLOCKS + NA_BLOCK - 1) / NA_BLOCK * NA_BLOCK;
    const int64_t min_chunk = 8 * NA_BLOCK;   // at most ~N / 2048 blocks for small trees
    if (chunk < min_chunk) chunk = min_chunk;
    const int G = (int)((N + chunk - 1) / chunk);
    // each launch reports its own status: an error left by the caller's earlier work is neither
    // reported as this call's nor cleared
    if (na_launch(na_mark_kernel, G, NA_BLOCK, s, *hier, *cam, chunk, scratch) != cudaSuccess ||
        na_launch(na_scan_kernel, 1, 1024, s, G, capacity, scratch, cut_offsets) != cudaSuccess ||
        na_launch(na_write_kernel, G, NA_BLOCK, s, *hier, *cam, chunk, (const uint32_t*)scratch, capacity, cut_ids,
                  cut_t) != cudaSuccess)
        return H3DGS_ERR_CUDA;
    if (total_out) {
        uint32_t tw[2];
        if (cudaMemcpyAsync(tw, scratch + NA_MASK_WORDS + NA_MAX_BLOCKS, sizeof(tw), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return H3DGS_ERR_CUDA;
        *total_out = (int64_t)tw[0] | ((int64_t)tw[1] << 32);
        if (*total_out > capacity) return H3DGS_ERR_CAPACITY;
    }
    return H3DGS_OK;
}
