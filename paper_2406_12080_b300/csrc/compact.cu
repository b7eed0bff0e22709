// Compaction of the hierarchy (Sec. 5.2) on the device.
//
// The paper's procedure visits the granularity levels tau_k = tau_min 2^k (k = 0, 1, ... while
// tau_k <= tau_max): it marks B_k, the bottom-most nodes of the union of the training views' cuts
// at tau_k, and removes every unmarked node strictly below B_k (the leaves start out marked).
// Granularity never decreases towards the root in any view (a parent's box contains its
// children's), so with e(n) = the maximum over the training views of eps(n):
//   * n is in B_k  <=>  (n is a leaf or e(n) < tau_k) and (n is the root or e(parent) >= tau_k),
//     i.e. B_k is the cut at tau_k of a view whose granularity is e;
//   * n lies strictly below a node of B_k  <=>  n is not the root and e(parent) < tau_k.
// Hence an interior non-root node is removed iff e(parent) < tau_last and no level has
// e(n) < tau_k <= e(parent), and every level can be evaluated for all nodes at once:
//   1. compact_emax_kernel   e(n) for every node, the views' centres staged in shared memory;
//   2. compact_keep_kernel   the keep test; a kept non-root node's key is its closest kept
//                            ancestor (its new parent), removed nodes and the root get 0xffffffff;
//   3. a stable radix sort by key drops those and groups each new parent's children in ascending
//      old index;
//   4. compact_groups_kernel first and end position of every node's group;
//   5. compact_level_kernel  once per level of the new tree, breadth-first numbering: a
//                            decoupled look-back scan over the level's child counts places every
//                            child right after the level;
//   6. compact_gather_kernel attribute rows and boxes of the kept nodes in the new order.
#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "lookback.cuh"

namespace h3dgs {
namespace {

constexpr int CP_BLOCK = 256;
constexpr int CP_CAMS = 512;        // camera centres staged in shared memory per round
constexpr int CP_MAX_LEVELS = 64;

struct Levels {
    int count;
    float tau[CP_MAX_LEVELS];
};

struct TmpMem {
    std::vector<void*> ptrs;
    ~TmpMem() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t n) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

// Camera centre and f = max(fx, fy) of every training view, in the cut's fp32 order.
__global__ void compact_cams_kernel(const h3dgs_camera* __restrict__ cams, int n, float4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float c[3];
    camera_centre(cams[i], c);
    out[i] = make_float4(c[0], c[1], c[2], fmaxf(cams[i].fx, cams[i].fy));
}

__global__ void __launch_bounds__(CP_BLOCK) compact_emax_kernel(const float4* __restrict__ rec, int64_t n,
                                                                const float4* __restrict__ cam_cf, int n_cams,
                                                                float* __restrict__ emax) {
    __shared__ float4 s_cam[CP_CAMS];
    const int64_t v = blockIdx.x * (int64_t)CP_BLOCK + threadIdx.x;
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
    if (v < n) {
        lo = rec[2 * v];
        hi = rec[2 * v + 1];
    }
    float e = __int_as_float(0xff800000);
    for (int c0 = 0; c0 < n_cams; c0 += CP_CAMS) {
        const int nc = min(CP_CAMS, n_cams - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < nc; i += CP_BLOCK) s_cam[i] = cam_cf[c0 + i];
        __syncthreads();
        for (int i = 0; i < nc; ++i) {
            const float4 c = s_cam[i];
            e = fmaxf(e, granularity(c.x, c.y, c.z, c.w, lo.x, lo.y, lo.z, hi.x, hi.y, hi.z));
        }
    }
    if (v < n) emax[v] = e;
}

__device__ __forceinline__ int32_t rec_parent(const float4* rec, int64_t v) { return __float_as_int(rec[2 * v].w); }

// Whether node v survives (see the file comment).
__device__ __forceinline__ bool keep_node(const float4* __restrict__ rec, const float* __restrict__ emax, int64_t v,
                                          const Levels& L) {
    if (L.count == 0) return true;
    const int32_t p = rec_parent(rec, v);
    if (p < 0 || __float_as_int(rec[2 * v + 1].w) == 0) return true;
    const float en = emax[v], ep = emax[p];
    if (ep >= L.tau[L.count - 1]) return true;
    for (int k = 0; k < L.count; ++k)
        if (en < L.tau[k] && L.tau[k] <= ep) return true;
    return false;
}

__global__ void __launch_bounds__(CP_BLOCK) compact_keep_kernel(const float4* __restrict__ rec, int64_t n,
                                                                const float* __restrict__ emax, Levels L,
                                                                uint32_t* __restrict__ key, uint32_t* flags) {
    for (int64_t v = blockIdx.x * (int64_t)CP_BLOCK + threadIdx.x; v < n; v += (int64_t)gridDim.x * CP_BLOCK) {
        uint32_t k = 0xffffffffu;
        if (v > 0 && keep_node(rec, emax, v, L)) {
            int64_t cur = v;
            int32_t p = rec_parent(rec, v);
            // parents precede their children, so the walk ends at the root (which is kept) at the latest
            while (true) {
                if (p < 0 || p >= cur) {
                    atomicOr(flags, FLAG_BAD_TOPOLOGY);
                    p = 0;
                    break;
                }
                if (keep_node(rec, emax, p, L)) break;
                cur = p;
                p = rec_parent(rec, p);
            }
            k = (uint32_t)p;
        }
        key[v] = k;
    }
}

__global__ void compact_groups_kernel(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ n_dev,
                                      int32_t* __restrict__ first, int32_t* __restrict__ end) {
    const int64_t m = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (i == 0 || keys[i - 1] != k) first[k] = (int32_t)i;
        if (i + 1 == m || keys[i + 1] != k) end[k] = (int32_t)(i + 1);
    }
}

// One level [s, e) of the new tree (new indices): numbers the children of its nodes from e on, in
// level order, and records the level's topology.  *next = the number of children.
__global__ void __launch_bounds__(CP_BLOCK) compact_level_kernel(int64_t s, int64_t e, const int32_t* __restrict__ first,
                                                                 const int32_t* __restrict__ end,
                                                                 const uint32_t* __restrict__ sorted_child,
                                                                 int32_t* __restrict__ old_of_new,
                                                                 int32_t* __restrict__ parent, int32_t* __restrict__ cstart,
                                                                 int32_t* __restrict__ ccount, Lookback lb,
                                                                 unsigned long long* __restrict__ next) {
    __shared__ uint32_t s_ticket;
    __shared__ unsigned long long s_warp[CP_BLOCK / 32];
    __shared__ unsigned long long s_prefix;
    const uint32_t b = lb_ticket(lb, &s_ticket);
    const int64_t j = s + (int64_t)b * CP_BLOCK + threadIdx.x;
    int32_t f = 0, c = 0;
    if (j < e) {
        const int32_t o = old_of_new[j];
        f = first[o];
        c = end[o] - f;
    }
    unsigned long long total;
    const unsigned long long ex = lb_block_scan<CP_BLOCK>((unsigned long long)c, s_warp, &total);
    const unsigned long long pre = lb_prefix(lb, b, total, &s_prefix);
    if (j < e) {
        const int64_t cb = e + (int64_t)(pre + ex);
        ccount[j] = c;
        cstart[j] = c ? (int32_t)cb : -1;
        for (int r = 0; r < c; ++r) {
            old_of_new[cb + r] = (int32_t)sorted_child[f + r];
            parent[cb + r] = (int32_t)j;
        }
    }
    if (b == gridDim.x - 1 && threadIdx.x == 0) *next = pre + total;
}

__global__ void compact_gather_kernel(int64_t m, const int32_t* __restrict__ old_of_new, h3dgs_hierarchy h,
                                      BuildOut out) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = old_of_new[j];
        for (int k = 0; k < 3; ++k) {
            out.mean[3 * j + k] = h.mean[3 * o + k];
            out.scale[3 * j + k] = h.scale[3 * o + k];
            out.box_min[3 * j + k] = h.box_min[3 * o + k];
            out.box_max[3 * j + k] = h.box_max[3 * o + k];
        }
        reinterpret_cast<float4*>(out.rot)[j] = reinterpret_cast<const float4*>(h.rot)[o];
        out.opacity[j] = h.opacity[o];
        const float4* src = reinterpret_cast<const float4*>(h.sh) + 12 * o;
        float4* dst = reinterpret_cast<float4*>(out.sh) + 12 * j;
#pragma unroll
        for (int q = 0; q < 12; ++q) dst[q] = src[q];
    }
}

int grid_for(int64_t n, int num_sms) {
    const int64_t want = (n + CP_BLOCK - 1) / CP_BLOCK;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms * 16));
}

}  // namespace

#define CR(expr)                              \
    do {                                      \
        cudaError_t e_ = (expr);              \
        if (e_ != cudaSuccess) return e_;     \
    } while (0)

cudaError_t compact_hierarchy(const h3dgs_hierarchy& h, const float4* rec, const h3dgs_camera* cams_host,
                              int n_cams, const float* levels, int n_levels, const BuildOut& out, int64_t capacity,
                              int32_t* old_index, int64_t* n_out, const SortWork& sw, int num_sms, cudaStream_t s) {
    if (n_levels < 0 || n_levels > CP_MAX_LEVELS || n_cams < 1) return cudaErrorInvalidValue;
    const int64_t N = h.n_nodes;
    Levels L;
    L.count = n_levels;
    for (int k = 0; k < n_levels; ++k) L.tau[k] = levels[k];
    TmpMem tm;
    h3dgs_camera* d_cams;
    float4* cam_cf;
    float* emax;
    uint32_t *key, *ka, *va, *kb, *vb, *counts;
    int32_t *first, *end, *o2n;
    unsigned long long* next;
    CR(tm.alloc(&d_cams, n_cams));
    CR(tm.alloc(&cam_cf, n_cams));
    CR(tm.alloc(&emax, N));
    CR(tm.alloc(&key, N));
    CR(tm.alloc(&ka, N));
    CR(tm.alloc(&va, N));
    CR(tm.alloc(&kb, N));
    CR(tm.alloc(&vb, N));
    CR(tm.alloc(&counts, 2));
    CR(tm.alloc(&first, N));
    CR(tm.alloc(&end, N));
    CR(tm.alloc(&o2n, N));
    CR(tm.alloc(&next, 1));

    CR(cudaMemcpyAsync(d_cams, cams_host, sizeof(h3dgs_camera) * n_cams, cudaMemcpyHostToDevice, s));
    compact_cams_kernel<<<(n_cams + 127) / 128, 128, 0, s>>>(d_cams, n_cams, cam_cf);
    CR(cudaGetLastError());
    compact_emax_kernel<<<(unsigned)((N + CP_BLOCK - 1) / CP_BLOCK), CP_BLOCK, 0, s>>>(rec, N, cam_cf, n_cams, emax);
    CR(cudaGetLastError());
    compact_keep_kernel<<<grid_for(N, num_sms), CP_BLOCK, 0, s>>>(rec, N, emax, L, key, sw.flags);
    CR(cudaGetLastError());

    // kept non-root nodes grouped by new parent, ascending old index within a group
    const uint32_t n32 = (uint32_t)N;
    CR(cudaMemcpyAsync(counts, &n32, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    int bits = 1;
    while (bits < 32 && (1ull << bits) < (unsigned long long)N) ++bits;
    bool in_a = true;
    CR(radix_sort_pairs(key, nullptr, ka, va, kb, vb, counts, N, bits, true, counts + 1, sw, &in_a, s));
    const uint32_t* skey = in_a ? ka : kb;
    const uint32_t* sval = in_a ? va : vb;
    uint32_t n_kept = 0;
    CR(cudaMemcpyAsync(&n_kept, counts + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CR(cudaStreamSynchronize(s));
    const int64_t M = 1 + (int64_t)n_kept;
    *n_out = M;
    if (M > capacity) return cudaSuccess;

    CR(cudaMemsetAsync(first, 0, sizeof(int32_t) * N, s));
    CR(cudaMemsetAsync(end, 0, sizeof(int32_t) * N, s));
    compact_groups_kernel<<<grid_for(n_kept, num_sms), CP_BLOCK, 0, s>>>(skey, counts + 1, first, end);
    CR(cudaGetLastError());

    const int32_t root_old = 0, root_parent = -1;
    CR(cudaMemcpyAsync(o2n, &root_old, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CR(cudaMemcpyAsync(out.parent, &root_parent, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    int64_t lo = 0, hi = 1;
    while (lo < hi) {
        const int64_t blocks = (hi - lo + CP_BLOCK - 1) / CP_BLOCK;
        if ((size_t)(LB_HEADER_WORDS + 2 * blocks) > sw.words) return cudaErrorInvalidValue;
        Lookback lb{reinterpret_cast<unsigned long long*>(sw.work + LB_HEADER_WORDS), sw.work, sw.flags};
        CR(cudaMemsetAsync(sw.work, 0, sizeof(uint32_t) * (LB_HEADER_WORDS + 2 * (size_t)blocks), s));
        compact_level_kernel<<<(unsigned)blocks, CP_BLOCK, 0, s>>>(lo, hi, first, end, sval, o2n, out.parent,
                                                                     out.child_start, out.child_count, lb, next);
        CR(cudaGetLastError());
        unsigned long long nc = 0;
        CR(cudaMemcpyAsync(&nc, next, sizeof(nc), cudaMemcpyDeviceToHost, s));
        CR(cudaStreamSynchronize(s));
        if (hi + (int64_t)nc > M) return cudaErrorInvalidValue;   // inconsistent topology
        lo = hi;
        hi += (int64_t)nc;
    }
    if (hi != M) return cudaErrorInvalidValue;
    compact_gather_kernel<<<grid_for(M, num_sms), CP_BLOCK, 0, s>>>(M, o2n, h, out);
    CR(cudaGetLastError());
    if (old_index) CR(cudaMemcpyAsync(old_index, o2n, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, s));
    return cudaStreamSynchronize(s);
}

}  // namespace h3dgs
