// Hierarchy residency (a0) and cut selection with interpolation weights (a1, a2).
//
// The cut follows the paper's constant-time-per-node rule (Sec. 4.2): node n is selected iff
// (eps(n) < tau or n is a leaf) and (n is the root or eps(parent) >= tau).  Because a parent's box
// contains its children's, eps never decreases towards the root, so this per-node test yields
// exactly one node on every root-to-leaf path.  The kernels scan all nodes (one 32-byte record
// each, plus the parent's record which is usually an L1/L2 hit for siblings) and test every
// camera of the batch against each node while it is in registers:
//   pass 1  one bit per (camera, node) in a mask, a count per (camera, block);
//   pass 2  scans of the counts (per camera over blocks, then over cameras);
//   pass 3  ordered compaction: ids in ascending order, t recomputed for the selected nodes.
#include "internal.cuh"
#include "lookback.cuh"

namespace h3dgs {

// ------------------------------------------------------------------------------------ a0

__global__ void pack_records_kernel(int64_t n, const float* __restrict__ bmin, const float* __restrict__ bmax,
                                    const int32_t* __restrict__ parent, const int32_t* __restrict__ ccount,
                                    float4* __restrict__ rec) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        rec[2 * v] = make_float4(bmin[3 * v], bmin[3 * v + 1], bmin[3 * v + 2], __int_as_float(parent[v]));
        rec[2 * v + 1] = make_float4(bmax[3 * v], bmax[3 * v + 1], bmax[3 * v + 2], __int_as_float(ccount[v]));
    }
}

cudaError_t launch_pack_records(const h3dgs_hierarchy& h, float4* rec, cudaStream_t s) {
    int64_t blocks = (h.n_nodes + 255) / 256;
    if (blocks > 65535 * 8) blocks = 65535 * 8;
    pack_records_kernel<<<(unsigned)blocks, 256, 0, s>>>(h.n_nodes, h.box_min, h.box_max, h.parent, h.child_count, rec);
    return cudaGetLastError();
}

__global__ void camera_setup_kernel(CamBatch b, DevCam* __restrict__ out) {
    griddep_launch_dependents();
    griddep_wait();
    if ((int)threadIdx.x < b.count) setup_camera(b, threadIdx.x, out);
}

cudaError_t launch_camera_setup(const CamBatch& b, const DevOpts*, DevCam* cams, cudaStream_t s) {
    return launch_dependent(camera_setup_kernel, dim3(1), dim3(CAM_BATCH), s, b, cams);
}

// ------------------------------------------------------------------------------------ a1 + a2

constexpr int CUT_BLOCK = 256;

__device__ __forceinline__ bool cut_test(const DevCam& cam, const float4 lo, const float4 hi, const float4 plo,
                                         const float4 phi, bool has_parent, float* en_out, float* ep_out) {
    const float en = granularity(cam, lo.x, lo.y, lo.z, hi.x, hi.y, hi.z);
    const bool leaf = __float_as_int(hi.w) == 0;
    float ep = __int_as_float(0x7f800000);
    bool parent_ok = true;
    // the parent's granularity only decides nodes that pass their own test (eps(n) < tau or a leaf);
    // the others are not selected whatever it is (ep_out is then not meaningful and not used)
    if (has_parent && ((en < cam.tau) || leaf)) {
        ep = granularity(cam, plo.x, plo.y, plo.z, phi.x, phi.y, phi.z);
        parent_ok = ep >= cam.tau;
    }
    *en_out = en;
    *ep_out = ep;
    return ((en < cam.tau) || leaf) && parent_ok;
}

// pass 1: selection bits and per-(camera, block) counts
__global__ void __launch_bounds__(CUT_BLOCK) cut_mark_kernel(const float4* __restrict__ rec, int64_t n,
                                                             const DevCam* __restrict__ cams, int n_cams,
                                                             int64_t chunk, int64_t words,
                                                             uint32_t* __restrict__ mask,
                                                             uint32_t* __restrict__ block_counts) {
    extern __shared__ uint32_t s_count[];  // [n_cams]
    for (int k = threadIdx.x; k < n_cams; k += blockDim.x) s_count[k] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t base = blockIdx.x * chunk;
    const int64_t end = min(base + chunk, n);
    for (int64_t v0 = base; v0 < end; v0 += CUT_BLOCK) {
        const int64_t v = v0 + threadIdx.x;
        const bool valid = v < end;
        float4 lo = make_float4(0, 0, 0, 0), hi = lo, plo = lo, phi = lo;
        int32_t p = -1;
        if (valid) {
            lo = __ldg(rec + 2 * v);
            hi = __ldg(rec + 2 * v + 1);
            p = __float_as_int(lo.w);
            if (p >= 0 && H3DGS_IN(p, n)) {
                plo = __ldg(rec + 2 * (int64_t)p);
                phi = __ldg(rec + 2 * (int64_t)p + 1);
            }
        }
        for (int k = 0; k < n_cams; ++k) {
            float en, ep;
            const bool sel = valid && cut_test(cams[k], lo, hi, plo, phi, p >= 0, &en, &ep);
            const uint32_t word = __ballot_sync(0xffffffffu, sel);
            if (lane == 0) {
                const int64_t w = (v - lane) >> 5;
                if (((v - lane) < end) || word) {
                    if (w < words) mask[(int64_t)k * words + w] = word;
                }
                if (word) atomicAdd(&s_count[k], (uint32_t)__popc(word));
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_cams; k += blockDim.x) block_counts[(int64_t)k * gridDim.x + blockIdx.x] = s_count[k];
}

// pass 2a: per camera, exclusive scan of the block counts (in place) and the camera total
__global__ void cut_scan_blocks_kernel(uint32_t* __restrict__ block_counts, int G, int64_t* __restrict__ cam_totals) {
    const int k = blockIdx.x;
    uint32_t* c = block_counts + (int64_t)k * G;
    __shared__ uint32_t s_part[1024];
    // each thread scans a contiguous segment
    const int per = (G + blockDim.x - 1) / blockDim.x;
    const int s0 = threadIdx.x * per, s1 = min(G, s0 + per);
    uint32_t sum = 0;
    for (int i = s0; i < s1; ++i) sum += c[i];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) { uint32_t x = s_part[i]; s_part[i] = run; run += x; }
        cam_totals[k] = run;
    }
    __syncthreads();
    uint32_t run = s_part[threadIdx.x];
    for (int i = s0; i < s1; ++i) { uint32_t x = c[i]; c[i] = run; run += x; }
}

// pass 2b: exclusive scan of the camera totals -> raw offsets; clamped offsets for the caller
__global__ void cut_scan_cams_kernel(int64_t* __restrict__ cam_totals, int n_cams, int64_t capacity,
                                     int64_t* __restrict__ cut_offsets, uint32_t* __restrict__ flags) {
    if (threadIdx.x != 0) return;
    int64_t run = 0;
    for (int k = 0; k < n_cams; ++k) {
        const int64_t x = cam_totals[k];
        cam_totals[k] = run;
        cut_offsets[k] = run < capacity ? run : capacity;
        run += x;
    }
    cam_totals[n_cams] = run;
    cut_offsets[n_cams] = run < capacity ? run : capacity;
    if (run > capacity) atomicOr(flags, FLAG_CUT_TRUNCATED);
}

// pass 3: ordered compaction and interpolation weights
__global__ void __launch_bounds__(CUT_BLOCK) cut_write_kernel(const float4* __restrict__ rec, int64_t n,
                                                              const DevCam* __restrict__ cams, int n_cams,
                                                              int64_t chunk, int64_t words,
                                                              const uint32_t* __restrict__ mask,
                                                              const uint32_t* __restrict__ block_offs,
                                                              const int64_t* __restrict__ cam_offs,
                                                              int64_t capacity, int32_t* __restrict__ cut_ids,
                                                              float* __restrict__ cut_t) {
    __shared__ uint32_t s_warp[CUT_BLOCK / 32];
    __shared__ int64_t s_run;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = blockIdx.x * chunk;
    const int64_t end = min(base + chunk, n);
    for (int k = 0; k < n_cams; ++k) {
        const DevCam& cam = cams[k];
        if (threadIdx.x == 0) s_run = cam_offs[k] + block_offs[(int64_t)k * gridDim.x + blockIdx.x];
        __syncthreads();
        for (int64_t v0 = base; v0 < end; v0 += CUT_BLOCK) {
            const int64_t v = v0 + threadIdx.x;
            const int64_t w = (v0 >> 5) + warp;
            const uint32_t word = (v0 + warp * 32 < end && w < words) ? mask[(int64_t)k * words + w] : 0u;
            const bool sel = (word >> lane) & 1u;
            if (lane == 0) s_warp[warp] = __popc(word);
            __syncthreads();
            uint32_t before = 0, total = 0;
            for (int i = 0; i < CUT_BLOCK / 32; ++i) {
                const uint32_t c = s_warp[i];
                before += (i < warp) ? c : 0u;
                total += c;
            }
            const int64_t pos = s_run + before + __popc(word & ((1u << lane) - 1u));
            if (sel && pos < capacity) {
                cut_ids[pos] = (int32_t)v;
                if (cut_t) {
                    const float4 lo = __ldg(rec + 2 * v), hi = __ldg(rec + 2 * v + 1);
                    const int32_t p = __float_as_int(lo.w);
                    float t = 0.0f;
                    if (p >= 0 && H3DGS_IN(p, n)) {
                        const float4 plo = __ldg(rec + 2 * (int64_t)p), phi = __ldg(rec + 2 * (int64_t)p + 1);
                        const float en = granularity(cam, lo.x, lo.y, lo.z, hi.x, hi.y, hi.z);
                        const float ep = granularity(cam, plo.x, plo.y, plo.z, phi.x, phi.y, phi.z);
                        t = parent_weight(cam.tau, en, ep);
                    }
                    cut_t[pos] = t;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) s_run += total;
            __syncthreads();
        }
    }
}

// One camera: a single pass with decoupled look-back.  Block b (ticket order) tests nodes
// [b T, (b + 1) T) (T = IPT CUT_BLOCK), IPT per thread at stride CUT_BLOCK (coalesced), counts the
// selected ones per (step, warp), obtains the count of all earlier blocks and writes its ids in
// ascending order with their weights.  The last block writes the offsets and the total.
constexpr int CS_IPT = 10;   // with at most 6 blocks of 256 per SM a 2M-node scan is one wave (8..16 measured, 10 fastest)
constexpr int CS_IPT_LARGE = 20;   // nodes per thread when the scan takes several waves (fewer, longer blocks)
constexpr int CS_GRP = 2;   // nodes whose loads are in flight together (2 measured fastest of 1, 2, 4, 8)
constexpr int CS_TILE = CUT_BLOCK * CS_IPT;
//
// Rows (CUT_BLOCK consecutive node ids, one step of a tile) that cannot hold a cut node are skipped
// without reading their records.  A node is only in the cut if eps(parent) >= tau (or it is the
// root).  Per row the upload stores the union box U of its nodes' parents and their largest side S
// (cut_row_bounds_kernel); every parent p then has eps(p) = f size_p / dist(c, box_p) <= f S / dist(c, U),
// since box_p lies inside U.  When that bound is below tau by a margin of 1e-4 (relative), far above
// the rounding of the bound and of the fp32 eps(p) the test would compute, no node of the row is
// selected.  A row holding any node of the cut or its ancestors is always read, so the scan reads at
// least what a root-down traversal visits; far chunks of a city lose most of their deep rows.
constexpr int CUT_ROW = CUT_BLOCK;

__global__ void __launch_bounds__(CUT_ROW) cut_row_bounds_kernel(const float4* __restrict__ rec, int64_t n,
                                                                 float4* __restrict__ rb) {
    __shared__ float s_r[CUT_ROW / 32][8];
    const float INF = __int_as_float(0x7f800000);
    float v[8] = {INF, INF, INF, 0.0f, -INF, -INF, -INF, 0.0f};   // U.lo, S, U.hi, no-skip flag
    const int64_t i = (int64_t)blockIdx.x * CUT_ROW + threadIdx.x;
    if (i < n) {
        const int32_t p = __float_as_int(__ldg(rec + 2 * i).w);
        if (p < 0 || p >= n) {   // the root (or an invalid parent): never skipped
            v[7] = 1.0f;
        } else {
            const float4 lo = __ldg(rec + 2 * (int64_t)p), hi = __ldg(rec + 2 * (int64_t)p + 1);
            const float s = fmaxf(fmaxf(fsub(hi.x, lo.x), fsub(hi.y, lo.y)), fsub(hi.z, lo.z));
            if (isnan(lo.x) || isnan(lo.y) || isnan(lo.z) || isnan(hi.x) || isnan(hi.y) || isnan(hi.z) || isnan(s))
                v[7] = 1.0f;
            v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = s; v[4] = hi.x; v[5] = hi.y; v[6] = hi.z;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float o = __shfl_xor_sync(0xffffffffu, v[k], off);
            v[k] = (k < 3) ? fminf(v[k], o) : fmaxf(v[k], o);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 8; ++k) s_r[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < CUT_ROW / 32; ++w)
            for (int k = 0; k < 8; ++k) v[k] = (k < 3) ? fminf(v[k], s_r[w][k]) : fmaxf(v[k], s_r[w][k]);
        rb[2 * blockIdx.x] = make_float4(v[0], v[1], v[2], v[3]);
        rb[2 * blockIdx.x + 1] = make_float4(v[4], v[5], v[6], v[7]);
    }
}

int64_t cut_row_count(int64_t n) { return (n + CUT_ROW - 1) / CUT_ROW; }

cudaError_t launch_cut_row_bounds(const float4* rec, int64_t n, float4* rb, cudaStream_t s) {
    const int64_t rows = cut_row_count(n);
    if (rows <= 0) return cudaSuccess;
    if (rows > 0x7fffffffLL) return cudaErrorInvalidValue;
    cut_row_bounds_kernel<<<(unsigned)rows, CUT_ROW, 0, s>>>(rec, n, rb);
    return cudaGetLastError();
}

template <int IPT>
__global__ void __launch_bounds__(CUT_BLOCK, 6) cut_single_kernel(const float4* __restrict__ rec, int64_t n,
                                                               const float4* __restrict__ rb,
                                                               const h3dgs_camera raw, int64_t capacity,
                                                               int32_t* __restrict__ cut_ids, float* __restrict__ cut_t,
                                                               int64_t* __restrict__ cut_offsets,
                                                               int64_t* __restrict__ cam_totals,
                                                               uint32_t* __restrict__ flags,
                                                               uint32_t* __restrict__ skipped, Lookback lb) {
    __shared__ uint32_t s_ticket;
    __shared__ unsigned long long s_slot, s_warp[CUT_BLOCK / 32];
    __shared__ uint32_t s_cnt[IPT][CUT_BLOCK / 32];
    __shared__ uint32_t s_word[IPT][CUT_BLOCK / 32];   // per (step, warp): ballot of the selected nodes
    __shared__ float s_tw[IPT][CUT_BLOCK];             // per (step, thread): the node's parent weight
    const uint32_t b = lb_ticket(lb, &s_ticket);
    const int64_t base = (int64_t)b * (CUT_BLOCK * IPT);
    if (base >= n) return;
    DevCam cam;   // only the centre, f and tau are used; derived as the set-up kernel does
    camera_centre(raw, cam.c);
    cam.f = fmaxf(raw.fx, raw.fy);
    cam.tau = raw.tau;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // rows of this tile whose bound test shows they hold no cut node (one bit per step, uniform)
    __shared__ uint32_t s_skip;
    if (warp == 0) {
        bool sk = false;
        const int64_t row = (int64_t)b * IPT + lane;
        if (rb && lane < IPT && base + (int64_t)lane * CUT_ROW < n) {
            const float4 u0 = __ldg(rb + 2 * row), u1 = __ldg(rb + 2 * row + 1);
            const float dx = fmaxf(fmaxf(u0.x - cam.c[0], cam.c[0] - u1.x), 0.0f);
            const float dy = fmaxf(fmaxf(u0.y - cam.c[1], cam.c[1] - u1.y), 0.0f);
            const float dz = fmaxf(fmaxf(u0.z - cam.c[2], cam.c[2] - u1.z), 0.0f);
            const float d2 = dx * dx + dy * dy + dz * dz;
            sk = u1.w == 0.0f && d2 > 0.0f && cam.f * u0.w < cam.tau * (1.0f - 1e-4f) * sqrtf(d2);
            if (sk && skipped) atomicAdd(skipped, (uint32_t)min((int64_t)CUT_ROW, n - (base + (int64_t)lane * CUT_ROW)));
        }
        const uint32_t m = __ballot_sync(0xffffffffu, sk);
        if (lane == 0) s_skip = m;
    }
    __syncthreads();
    const uint32_t skip = s_skip;
    {
        // CS_GRP nodes at a time: their records are all requested, then their parents' records, so a
        // thread keeps 2 CS_GRP loads in flight instead of one dependent pair
#pragma unroll
        for (int g = 0; g < IPT; g += CS_GRP) {
            float4 lo[CS_GRP], hi[CS_GRP], plo[CS_GRP], phi[CS_GRP];
#pragma unroll
            for (int k = 0; k < CS_GRP; ++k) {
                const int64_t v = base + (g + k) * CUT_BLOCK + threadIdx.x;
                const bool rd = v < n && !((skip >> (g + k)) & 1u);
                lo[k] = rd ? __ldg(rec + 2 * v) : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
                hi[k] = rd ? __ldg(rec + 2 * v + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < CS_GRP; ++k) {
                const int32_t p = __float_as_int(lo[k].w);
                const bool pin = p >= 0 && H3DGS_IN(p, n);
                plo[k] = pin ? __ldg(rec + 2 * (int64_t)p) : lo[k];
                phi[k] = pin ? __ldg(rec + 2 * (int64_t)p + 1) : hi[k];
            }
#pragma unroll
            for (int k = 0; k < CS_GRP; ++k) {
                const int q = g + k;
                const int64_t v = base + q * CUT_BLOCK + threadIdx.x;
                const int32_t p = __float_as_int(lo[k].w);
                bool sel = false;
                float tw = 0.0f;
                if (v < n && !((skip >> q) & 1u)) {
                    float en, ep;
                    sel = cut_test(cam, lo[k], hi[k], plo[k], phi[k], p >= 0, &en, &ep);
                    if (sel && p >= 0) tw = parent_weight(cam.tau, en, ep);
                }
                const uint32_t word = __ballot_sync(0xffffffffu, sel);
                s_tw[q][threadIdx.x] = tw;
                if (lane == 0) {
                    s_cnt[q][warp] = __popc(word);
                    s_word[q][warp] = word;
                }
            }
        }
    }
    __syncthreads();
    // exclusive scan of the (step, warp) counts in step-major order = ascending node order
    unsigned long long mine = 0;
    if (threadIdx.x < IPT * (CUT_BLOCK / 32)) mine = (&s_cnt[0][0])[threadIdx.x];
    unsigned long long agg;
    const unsigned long long ex = lb_block_scan<CUT_BLOCK>(mine, s_warp, &agg);
    if (threadIdx.x < IPT * (CUT_BLOCK / 32)) (&s_cnt[0][0])[threadIdx.x] = (uint32_t)ex;
    // a block with nothing to write publishes its count without waiting for its prefix (the block
    // holding the last node still waits: it writes the offsets and the total)
    if (agg == 0 && base + (int64_t)CUT_BLOCK * IPT < n) {
        lb_publish(lb, b, 0ull);
        return;
    }
    const unsigned long long prefix = lb_prefix(lb, b, agg, &s_slot);   // ends with a barrier
    const uint32_t lmask = (1u << lane) - 1u;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const uint32_t word = s_word[q][warp];
        if ((word >> lane) & 1u) {
            const int64_t pos = (int64_t)(prefix + s_cnt[q][warp]) + __popc(word & lmask);
            if (pos < capacity) {
                cut_ids[pos] = (int32_t)(base + q * CUT_BLOCK + threadIdx.x);
                if (cut_t) cut_t[pos] = s_tw[q][threadIdx.x];
            }
        }
    }
    if (base + (CUT_BLOCK * IPT) >= n && threadIdx.x == 0) {   // the last block: offsets and total
        const int64_t total = (int64_t)(prefix + agg);
        cam_totals[0] = 0;
        cam_totals[1] = total;
        cut_offsets[0] = 0;
        cut_offsets[1] = total < capacity ? total : capacity;
        if (total > capacity) atomicOr(flags, FLAG_CUT_TRUNCATED);
    }
}

size_t cut_single_work_words(int64_t n) {
    return LB_HEADER_WORDS + lb_body_words((n + CS_TILE - 1) / CS_TILE);
}

cudaError_t launch_cut(const DevHier& h, const DevCam* cams, int n_cams, const CutWork& w, int32_t* cut_ids,
                       float* cut_t, int64_t* cut_offsets, int64_t capacity, uint32_t* flags, cudaStream_t s) {
    if (n_cams == 1 && w.lb_work) {
        // one wave of small tiles where they all fit (at most 6 blocks of 256 per SM), else longer tiles
        const bool large = (h.n + CS_TILE - 1) / CS_TILE > 6 * (int64_t)w.num_sms;
        const int64_t tile = (int64_t)CUT_BLOCK * (large ? CS_IPT_LARGE : CS_IPT);
        const int64_t blocks = (h.n + tile - 1) / tile;
        const size_t words = LB_HEADER_WORDS + lb_body_words(blocks);
        if ((int64_t)words > w.lb_words) return cudaErrorInvalidValue;
        cudaError_t e = cudaMemsetAsync(w.lb_work, 0, sizeof(uint32_t) * words, s);
        if (e != cudaSuccess) return e;
        // grouped prefix when every block is resident (at most 6 blocks of 256 per SM)
        const Lookback lb = lb_make(w.lb_work, blocks, blocks <= 6 * (int64_t)w.num_sms, flags);
        if (large)
            cut_single_kernel<CS_IPT_LARGE><<<(unsigned)blocks, CUT_BLOCK, 0, s>>>(
                h.rec, h.n, h.row_bound, w.cam0, capacity, cut_ids, cut_t, cut_offsets, w.cam_totals, flags,
                w.skipped_nodes, lb);
        else
            cut_single_kernel<CS_IPT><<<(unsigned)blocks, CUT_BLOCK, 0, s>>>(
                h.rec, h.n, h.row_bound, w.cam0, capacity, cut_ids, cut_t, cut_offsets, w.cam_totals, flags,
                w.skipped_nodes, lb);
        return cudaGetLastError();
    }
    const size_t smem = sizeof(uint32_t) * (size_t)n_cams;
    cut_mark_kernel<<<w.blocks, CUT_BLOCK, smem, s>>>(h.rec, h.n, cams, n_cams, w.chunk, w.words, w.mask,
                                                      w.block_counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cut_scan_blocks_kernel<<<n_cams, 256, 0, s>>>(w.block_counts, w.blocks, w.cam_totals);
    cut_scan_cams_kernel<<<1, 32, 0, s>>>(w.cam_totals, n_cams, capacity, cut_offsets, flags);
    cut_write_kernel<<<w.blocks, CUT_BLOCK, 0, s>>>(h.rec, h.n, cams, n_cams, w.chunk, w.words, w.mask, w.block_counts,
                                                    w.cam_totals, capacity, cut_ids, cut_t);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ a1 + a2, traversal
//
// One camera on a large tree: a persistent grid descends from the root level by level and reads only
// the records of the nodes it visits, the cut and its ancestors, instead of all N.  The descent gives
// exactly the scan's set: a frontier node's parent was expanded (eps(parent) >= tau, not a leaf), so it
// is in the cut iff eps(n) < tau or it is a leaf; and eps does not decrease towards the root (nested
// boxes, fixed fp32 order), so a node whose parent passes the test has every ancestor passing it too.
// Cut nodes set their bit in a mark array and store their parent weight per node; an ordered
// compaction of the marks then writes the ids in ascending order (the consolidated trees are not
// globally breadth-first, so a level's ids do not follow the previous level's).  Levels are separated
// by a grid barrier of bounded waits; the launch is cooperative, so every block is resident.

constexpr int TR_BLOCK = 256;
constexpr int TR_SPIN_LIMIT = 1 << 22;   // polls of one barrier wait before it gives up (flagged)

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier: arrivals counted in bar[0], the release published as a new generation in bar[1].
// Bounded: a wait that gives up sets FLAG_WAIT_TIMEOUT (the cut is then invalid) and goes on.  Returns,
// uniformly over the block, whether any wait of the launch has given up so far.
__device__ __forceinline__ bool grid_sync_bounded(uint32_t* bar, uint32_t nblocks, uint32_t& gen, uint32_t* flags) {
    __shared__ uint32_t s_failed;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t arrived = atomicAdd(bar, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(bar + 1), "r"(gen + 1) : "memory");
        } else {
            uint32_t g = gen;
            int spins = 0;
            while (spins < TR_SPIN_LIMIT) {
                g = ld_acquire_u32(bar + 1);
                if (g != gen) break;
                if (++spins > 64) __nanosleep(100);
            }
            if (g == gen) atomicOr(flags, FLAG_WAIT_TIMEOUT);
        }
        gen += 1;
        s_failed = ld_acquire_u32(flags) & FLAG_WAIT_TIMEOUT;
    }
    __syncthreads();
    return s_failed != 0;
}

constexpr int TR_IPT = 4;                       // frontier entries per thread per round
constexpr int TR_TILE = TR_BLOCK * TR_IPT;

// Visit up to TR_IPT nodes per thread: all their loads are issued first; a cut node sets its mark (one
// atomic OR per mark word per warp) and its parent weight; an expanded node reports its child range.
// Returns the thread's number of children.
__device__ __forceinline__ uint32_t tr_visit(const TravArgs& a, const DevCam& cam, const uint32_t (&v)[TR_IPT],
                                             const float (&ep)[TR_IPT], int (&cnt)[TR_IPT], int32_t (&cs)[TR_IPT],
                                             float (&en)[TR_IPT], int lane) {
    float4 lo[TR_IPT], hi[TR_IPT];
    bool ok[TR_IPT];
#pragma unroll
    for (int k = 0; k < TR_IPT; ++k) {
        ok[k] = v[k] < (uint64_t)a.n && H3DGS_IN(v[k], a.n);
        lo[k] = ok[k] ? __ldg(a.rec + 2 * (int64_t)v[k]) : make_float4(0.f, 0.f, 0.f, 0.f);
        hi[k] = ok[k] ? __ldg(a.rec + 2 * (int64_t)v[k] + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        cs[k] = ok[k] ? __ldg(a.child_start + v[k]) : 0;
    }
    uint32_t mine = 0;
#pragma unroll
    for (int k = 0; k < TR_IPT; ++k) {
        cnt[k] = 0;
        en[k] = 0.0f;
        bool is_cut = false;
        if (ok[k]) {
            en[k] = granularity(cam, lo[k].x, lo[k].y, lo[k].z, hi[k].x, hi[k].y, hi[k].z);
            const int cc = __float_as_int(hi[k].w);
            if (en[k] < cam.tau || cc == 0) {
                is_cut = true;
                a.tnode[v[k]] = parent_weight(cam.tau, en[k], ep[k]);   // the root (ep = +inf): 0
            } else {
                cnt[k] = cc;
            }
        }
        const uint32_t key = is_cut ? (v[k] >> 5) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        const uint32_t bits = __reduce_or_sync(peers, is_cut ? (1u << (v[k] & 31)) : 0u);
        if (is_cut && lane == __ffs(peers) - 1) atomicOr(a.mark + key, bits);
        mine += (uint32_t)cnt[k];
    }
    return mine;
}

constexpr int TR_CBUF = 2 * TR_TILE;            // children a block keeps in shared memory per round

__global__ void __launch_bounds__(TR_BLOCK) cut_traverse_kernel(TravArgs a, const h3dgs_camera raw) {
    __shared__ unsigned long long s_warp[TR_BLOCK / 32];
    __shared__ uint32_t s_base;
    __shared__ uint32_t s_cid[TR_CBUF];
    __shared__ float s_ceps[TR_CBUF];
    DevCam cam;   // only the centre, f and tau are used; derived as the set-up kernel does
    camera_centre(raw, cam.c);
    cam.f = fmaxf(raw.fx, raw.fy);
    cam.tau = raw.tau;
    const float INF = __int_as_float(0x7f800000);
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * TR_TILE;
    uint32_t gen = 0;
    // Each step takes the frontier (nodes whose parent was expanded, of any depth) and visits them and,
    // inside the block, their children: only the grandchildren go to the next step's frontier, so a step
    // descends two levels and one grid barrier separates steps.
    for (int step = 0; step < TR_MAX_LEVELS; ++step) {
        const uint32_t m = step == 0 ? 1u : ld_acquire_u32(a.level_count + step);
        if (m == 0) break;
        const uint32_t mm = (int64_t)m > a.cap ? (uint32_t)a.cap : m;
        const bool odd = step & 1;
        const uint32_t* f_in = odd ? a.front[1] : a.front[0];
        const float* e_in = odd ? a.feps[1] : a.feps[0];
        uint32_t* f_out = odd ? a.front[0] : a.front[1];
        float* e_out = odd ? a.feps[0] : a.feps[1];
        uint32_t* out_count = a.level_count + step + 1;
        for (uint64_t i0 = (uint64_t)blockIdx.x * TR_TILE; i0 < mm; i0 += stride) {   // uniform per block
            uint32_t v[TR_IPT];
            float ep[TR_IPT];
#pragma unroll
            for (int k = 0; k < TR_IPT; ++k) {
                const uint64_t i = i0 + (uint64_t)k * TR_BLOCK + threadIdx.x;
                v[k] = 0xffffffffu;
                ep[k] = INF;
                if (i < mm) {
                    // written by other blocks during the previous step: read at L2, past any stale L1 line
                    v[k] = step == 0 ? 0u : __ldcg(f_in + i);
                    ep[k] = step == 0 ? INF : __ldcg(e_in + i);
                }
            }
            int cnt[TR_IPT];
            int32_t cs[TR_IPT];
            float en[TR_IPT];
            uint32_t mine = tr_visit(a, cam, v, ep, cnt, cs, en, lane);
            // children: the first TR_CBUF of the block into shared memory, any more to the next frontier
            unsigned long long total;
            unsigned long long pos = lb_block_scan<TR_BLOCK>(mine, s_warp, &total);
            const uint32_t spill = total > (unsigned long long)TR_CBUF ? (uint32_t)(total - TR_CBUF) : 0u;
            if (threadIdx.x == 0) s_base = spill ? atomicAdd(out_count, spill) : 0u;
            __syncthreads();
#pragma unroll
            for (int k = 0; k < TR_IPT; ++k)
                for (int c = 0; c < cnt[k]; ++c, ++pos) {
                    if (pos < (unsigned long long)TR_CBUF) {
                        s_cid[pos] = (uint32_t)(cs[k] + c);
                        s_ceps[pos] = en[k];
                    } else {
                        const uint64_t g = (uint64_t)s_base + (pos - TR_CBUF);
                        if (g < (uint64_t)a.cap) {
                            f_out[g] = (uint32_t)(cs[k] + c);
                            e_out[g] = en[k];
                        }
                    }
                }
            if (threadIdx.x == 0 && spill && (uint64_t)s_base + spill > (uint64_t)a.cap)
                atomicOr(a.flags, FLAG_CUT_TRUNCATED);
            __syncthreads();
            // the children kept in shared memory, TR_IPT per thread per round (consecutive ids per warp)
            const uint32_t nc = total < (unsigned long long)TR_CBUF ? (uint32_t)total : (uint32_t)TR_CBUF;
            if (threadIdx.x == 0 && nc) atomicAdd(a.inner, nc);   // nodes visited without a frontier entry
            for (uint32_t r0 = 0; r0 < nc; r0 += TR_TILE) {   // uniform per block
#pragma unroll
                for (int k = 0; k < TR_IPT; ++k) {
                    const uint32_t q = r0 + k * TR_BLOCK + threadIdx.x;
                    v[k] = q < nc ? s_cid[q] : 0xffffffffu;
                    ep[k] = q < nc ? s_ceps[q] : INF;
                }
                mine = tr_visit(a, cam, v, ep, cnt, cs, en, lane);
                unsigned long long tot2;
                unsigned long long p2 = lb_block_scan<TR_BLOCK>(mine, s_warp, &tot2);
                if (threadIdx.x == 0) s_base = tot2 ? atomicAdd(out_count, (uint32_t)tot2) : 0u;
                __syncthreads();
                p2 += s_base;
                if (threadIdx.x == 0 && (uint64_t)s_base + tot2 > (uint64_t)a.cap) atomicOr(a.flags, FLAG_CUT_TRUNCATED);
#pragma unroll
                for (int k = 0; k < TR_IPT; ++k)
                    for (int c = 0; c < cnt[k]; ++c, ++p2)
                        if (p2 < (uint64_t)a.cap) {
                            f_out[p2] = (uint32_t)(cs[k] + c);
                            e_out[p2] = en[k];
                        }
                __syncthreads();   // s_base and s_warp are reused
            }
        }
        // a barrier that gave up invalidates the cut (flagged): stop instead of waiting at every later step
        if (grid_sync_bounded(a.bar, gridDim.x, gen, a.flags)) break;
        if (step == TR_MAX_LEVELS - 1 && threadIdx.x == 0 && blockIdx.x == 0 &&
            ld_acquire_u32(a.level_count + step + 1) != 0)
            atomicOr(a.flags, FLAG_CUT_TRUNCATED);   // deeper than the step table: the cut is incomplete
    }
}

// Ordered compaction of the marks.  A block covers TC_TILE consecutive mark words, each warp TC_ROUNDS
// rounds of 32 words (lane i holds word i of the round: coalesced loads).  The counts give every round
// its output range (warp scans, a block scan over the warps, a single-pass look-back over the blocks);
// the ids of a round are then written 32 consecutive slots at a time: the lane of slot s finds the
// word holding it (binary search over the lanes' prefixes by shuffles) and its bit (__fns), so the
// stores of a warp are contiguous.  The words are cleared for the next traversal.
constexpr int TC_ROUNDS = 4;
constexpr int TC_TILE = TR_BLOCK * TC_ROUNDS;   // mark words per block

__global__ void __launch_bounds__(TR_BLOCK) cut_compact_kernel(uint32_t* __restrict__ mark,
                                                               const float* __restrict__ tnode, int64_t n,
                                                               int64_t capacity, int32_t* __restrict__ cut_ids,
                                                               float* __restrict__ cut_t,
                                                               int64_t* __restrict__ cut_offsets,
                                                               int64_t* __restrict__ cam_totals,
                                                               uint32_t* __restrict__ flags, Lookback lb) {
    __shared__ uint32_t s_ticket;
    __shared__ unsigned long long s_slot, s_warp[TR_BLOCK / 32];
    const uint32_t b = lb_ticket(lb, &s_ticket);
    const int64_t words = (n + 31) / 32;
    if ((int64_t)b * TC_TILE >= words) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t wbase = (int64_t)b * TC_TILE + (int64_t)warp * 32 * TC_ROUNDS;
    uint32_t wv[TC_ROUNDS], incl[TC_ROUNDS], rtot[TC_ROUNDS];
    uint32_t mine = 0;
#pragma unroll
    for (int r = 0; r < TC_ROUNDS; ++r) {
        const int64_t w = wbase + r * 32 + lane;
        wv[r] = w < words ? mark[w] : 0u;
        incl[r] = __popc(wv[r]);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl[r], off);
            if (lane >= off) incl[r] += y;
        }
        rtot[r] = __shfl_sync(0xffffffffu, incl[r], 31);
        mine += rtot[r];
    }
    // block scan over the warps' totals (lane 0 of each warp contributes), then the look-back
    unsigned long long agg;
    const unsigned long long before = lb_block_scan<TR_BLOCK>(lane == 0 ? mine : 0u, s_warp, &agg);
    const unsigned long long wpre = __shfl_sync(0xffffffffu, before, 0);
    const unsigned long long prefix = lb_prefix(lb, b, agg, &s_slot);   // ends with a barrier
    int64_t base = (int64_t)(prefix + wpre);
#pragma unroll
    for (int r = 0; r < TC_ROUNDS; ++r) {
        const uint32_t ex = incl[r] - __popc(wv[r]);   // this lane's first slot within the round
        for (uint32_t s0 = 0; s0 < rtot[r]; s0 += 32) {
            const uint32_t slot = s0 + lane;
            // owner: the last lane whose exclusive prefix is <= slot
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t e = __shfl_sync(0xffffffffu, ex, lo + step);
                if (e <= slot) lo += step;
            }
            const uint32_t wo = __shfl_sync(0xffffffffu, wv[r], lo);
            const uint32_t eo = __shfl_sync(0xffffffffu, ex, lo);
            if (slot < rtot[r]) {
                const int bit = (int)__fns(wo, 0u, (int)(slot - eo) + 1);   // -1 if absent (never)
                const int64_t v = (wbase + r * 32 + lo) * 32 + bit;
                const int64_t pos = base + slot;
                if (pos < capacity && bit >= 0 && v < n && H3DGS_IN(v, n)) {
                    cut_ids[pos] = (int32_t)v;
                    if (cut_t) cut_t[pos] = tnode[v];
                }
            }
        }
        base += rtot[r];
        const int64_t w = wbase + r * 32 + lane;
        if (w < words && wv[r]) mark[w] = 0u;
    }
    if ((int64_t)(b + 1) * TC_TILE >= words && threadIdx.x == 0) {   // the last block: offsets and total
        const int64_t total = (int64_t)(prefix + agg);
        cam_totals[0] = 0;
        cam_totals[1] = total;
        cut_offsets[0] = 0;
        cut_offsets[1] = total < capacity ? total : capacity;
        if (total > capacity) atomicOr(flags, FLAG_CUT_TRUNCATED);
    }
}

size_t cut_traverse_work_words(int64_t n) {
    return LB_HEADER_WORDS + lb_body_words(std::max<int64_t>(1, ((n + 31) / 32 + TC_TILE - 1) / TC_TILE));
}

cudaError_t launch_cut_traverse(const TravArgs& a, const h3dgs_camera& cam, int grid, uint32_t* lb_work,
                                int64_t lb_words, int32_t* cut_ids, float* cut_t, int64_t* cut_offsets,
                                int64_t* cam_totals, int64_t capacity, cudaStream_t s) {
    const int64_t words = (a.n + 31) / 32;
    const int64_t cblocks = std::max<int64_t>(1, (words + TC_TILE - 1) / TC_TILE);
    const size_t lw = LB_HEADER_WORDS + lb_body_words(cblocks);
    if ((int64_t)lw > lb_words) return cudaErrorInvalidValue;
    // level counts and the barrier words are zero before the descent, the look-back words before the compaction
    cudaError_t e = cudaMemsetAsync(a.level_count, 0, sizeof(uint32_t) * TR_LEVEL_WORDS, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(lb_work, 0, sizeof(uint32_t) * lw, s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(TR_BLOCK);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, cut_traverse_kernel, a, cam);
    if (e != cudaSuccess) return e;
    const Lookback lb = lb_make(lb_work, cblocks, false, a.flags);
    cut_compact_kernel<<<(unsigned)cblocks, TR_BLOCK, 0, s>>>(a.mark, a.tnode, a.n, capacity, cut_ids, cut_t,
                                                            cut_offsets, cam_totals, a.flags, lb);
    return cudaGetLastError();
}

int cut_traverse_grid(int num_sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cut_traverse_kernel, TR_BLOCK, 0) != cudaSuccess ||
        per_sm < 1)
        return 0;
    return per_sm * num_sms;
}

H3DGS_CHECK_READER(check_read_cut)

}  // namespace h3dgs
