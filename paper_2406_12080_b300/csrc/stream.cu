// Streamed (out-of-core) rendering (Sec. 6.3: the cut is updated every few frames by transferring
// the nodes it needs from CPU RAM to the GPU, and a cleanup runs every 100 frames).
//
// Only the 32-byte cut records (boxes and topology) are resident for every node; node attributes
// stay in page-locked host memory and a device cache holds the rows of the nodes the recent cuts
// needed.  slot_of[node] is the node's cache row (-1: absent), node_of[slot] the row's node (-1:
// free), stamp[slot] the frame of the last update that needed it.  An update
//   1. stream_need_kernel    marks the cut's nodes and the parents of entries with t != 0: a
//                            resident one gets the new stamp, an absent one is claimed once
//                            (slot_of = -2) and appended to the transfer list;
//   2. stream_assign_kernel  gives the listed nodes free rows (a stack of free rows);
//   3. stream_pop_kernel     updates the free count and records the number transferred;
//   4. stream_gather_kernel  copies the listed nodes' rows from host memory, one warp per node,
//                            reading the host arrays through their device mapping (the copy runs
//                            on the GPU over the host link, no host-side gather).
// A cleanup returns to the free stack every row whose stamp is older than frame - max_age.
// The render reads attributes through slot_of (DevHier::row_of); values are the same floats as
// in host memory, so a streamed frame equals the resident one bit for bit.
#include <algorithm>

#include "internal.cuh"

namespace h3dgs {
namespace {

constexpr int ST_BLOCK = 256;

__global__ void stream_init_kernel(StreamState st) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < st.n_nodes; i += stride) st.slot_of[i] = -1;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < st.cap; s += stride) {
        st.node_of[s] = -1;
        st.stamp[s] = 0;
        st.free_list[s] = (int32_t)(st.cap - 1 - s);   // popped from the end: row 0 first
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st.count[0] = (uint32_t)st.cap;
        st.count[1] = st.count[2] = st.count[3] = 0;
    }
}

__device__ __forceinline__ void need_node(const StreamState& st, int32_t x, int32_t frame) {
    const int32_t s = *reinterpret_cast<volatile const int32_t*>(st.slot_of + x);
    if (s >= 0) {
        st.stamp[s] = frame;
        return;
    }
    if (s == -1 && atomicCAS(st.slot_of + x, -1, -2) == -1) st.missing[atomicAdd(st.count + 1, 1u)] = x;
}

__global__ void __launch_bounds__(ST_BLOCK) stream_need_kernel(StreamState st, const int32_t* __restrict__ parent,
                                                               int n_cams, const int32_t* __restrict__ cut_ids,
                                                               const float* __restrict__ cut_t,
                                                               const int64_t* __restrict__ cut_offsets, int32_t frame) {
    const int64_t M = cut_offsets[n_cams];
    for (int64_t m = blockIdx.x * (int64_t)ST_BLOCK + threadIdx.x; m < M; m += (int64_t)gridDim.x * ST_BLOCK) {
        const int32_t x = cut_ids[m];
        need_node(st, x, frame);
        if (cut_t && cut_t[m] != 0.0f) {
            const int32_t p = parent[x];
            if (p >= 0) need_node(st, p, frame);
        }
    }
}

__global__ void __launch_bounds__(ST_BLOCK) stream_assign_kernel(StreamState st, int32_t frame, uint32_t* flags) {
    const uint32_t n_miss = st.count[1], n_free = st.count[0];
    for (int64_t i = blockIdx.x * (int64_t)ST_BLOCK + threadIdx.x; i < n_miss; i += (int64_t)gridDim.x * ST_BLOCK) {
        const int32_t x = st.missing[i];
        if (i < n_free) {
            const int32_t slot = st.free_list[n_free - 1 - i];
            st.slot_of[x] = slot;
            st.node_of[slot] = x;
            st.stamp[slot] = frame;
        } else {
            st.slot_of[x] = -1;
            atomicOr(flags, FLAG_CACHE_FULL);
        }
    }
}

__global__ void stream_pop_kernel(StreamState st) {
    const uint32_t n_miss = st.count[1], n_free = st.count[0];
    const uint32_t used = min(n_miss, n_free);
    st.count[0] = n_free - used;
    st.count[2] = used;
    st.count[3] = n_miss;
    st.count[1] = 0;
}

__global__ void __launch_bounds__(ST_BLOCK) stream_gather_kernel(StreamState st) {
    const uint32_t used = st.count[2];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (ST_BLOCK / 32);
    for (int64_t i = (blockIdx.x * (int64_t)ST_BLOCK + threadIdx.x) >> 5; i < used; i += warps) {
        const int64_t x = st.missing[i];
        const int64_t slot = st.slot_of[x];
        const float* src = st.h_sh + 48 * x;
        float* dst = st.sh + 48 * slot;
        dst[lane] = src[lane];
        if (lane < 16) dst[32 + lane] = src[32 + lane];
        if (lane < 3) {
            st.mean[3 * slot + lane] = st.h_mean[3 * x + lane];
            st.scale[3 * slot + lane] = st.h_scale[3 * x + lane];
        }
        if (lane < 4) st.rot[4 * slot + lane] = st.h_rot[4 * x + lane];
        if (lane == 0) st.opacity[slot] = st.h_opacity[x];
    }
}

__global__ void __launch_bounds__(ST_BLOCK) stream_cleanup_kernel(StreamState st, int32_t frame, int32_t max_age) {
    for (int64_t s = blockIdx.x * (int64_t)ST_BLOCK + threadIdx.x; s < st.cap; s += (int64_t)gridDim.x * ST_BLOCK) {
        const int32_t x = st.node_of[s];
        if (x >= 0 && (int64_t)frame - st.stamp[s] > max_age) {
            st.slot_of[x] = -1;
            st.node_of[s] = -1;
            st.free_list[atomicAdd(st.count, 1u)] = (int32_t)s;
        }
    }
}

int grid_of(int64_t n, int num_sms) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + ST_BLOCK - 1) / ST_BLOCK, (int64_t)num_sms * 16));
}

}  // namespace

cudaError_t stream_init(const StreamState& st, int num_sms, cudaStream_t s) {
    stream_init_kernel<<<grid_of(std::max(st.n_nodes, st.cap), num_sms), ST_BLOCK, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t stream_update(const StreamState& st, const int32_t* parent, int n_cams, const int32_t* cut_ids,
                          const float* cut_t, const int64_t* cut_offsets, int32_t frame, uint32_t* flags, int num_sms,
                          cudaStream_t s) {
    const int grid = num_sms * 8;
    stream_need_kernel<<<grid, ST_BLOCK, 0, s>>>(st, parent, n_cams, cut_ids, cut_t, cut_offsets, frame);
    stream_assign_kernel<<<grid, ST_BLOCK, 0, s>>>(st, frame, flags);
    stream_pop_kernel<<<1, 1, 0, s>>>(st);
    stream_gather_kernel<<<grid, ST_BLOCK, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t stream_cleanup(const StreamState& st, int32_t frame, int32_t max_age, int num_sms, cudaStream_t s) {
    stream_cleanup_kernel<<<grid_of(st.cap, num_sms), ST_BLOCK, 0, s>>>(st, frame, max_age);
    return cudaGetLastError();
}

}  // namespace h3dgs
