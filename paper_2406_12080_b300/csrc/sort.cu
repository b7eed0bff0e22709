// Binning (a5) and tile ranges (a6), plus the device radix sort they and the hierarchy builder use.
//
// Tile lists come out in (depth, cut position) order without any per-tile sort:
//   1. the visible splats are sorted by their fp32 depth bits (stable LSD radix, input in cut
//      order, so equal depths stay in cut-position order; culled splats are dropped by the first
//      pass);
//   2. a scan of the per-splat tile counts in that order gives every splat its first pair slot;
//   3. every splat writes one (tile id, cut position) pair per covered tile;
//   4. the pairs are sorted stably by tile id (ceil(log2 tiles) bits, 2 passes at 1080p), which
//      keeps each tile's entries in depth order;
//   5. tile ranges are read off the sorted tile ids.
//
// The radix sort is an LSD "onesweep" sort with 8-bit digits: one kernel computes the digit
// histograms of every pass, then one kernel per pass ranks a tile of keys stably in shared memory,
// publishes the tile's digit counts, obtains the counts of all earlier tiles by decoupled look-back
// and scatters the keys, staged by digit so that the writes come out in runs.  Tiles take their
// index from a ticket counter, so every tile a block waits for belongs to a block that is already
// running; each wait is bounded and sets a device flag if it gives up.  All element counts live in
// device memory, so no launch depends on the host.
#include <algorithm>

#include "internal.cuh"

namespace h3dgs {

// ------------------------------------------------------------------------------ radix sort

constexpr int OS_THREADS = 256;                 // one thread per digit in the look-back
constexpr int OS_WARPS = OS_THREADS / 32;
constexpr int OS_IPT = 15;                      // keys per thread
constexpr int OS_TILE = OS_THREADS * OS_IPT;    // 3840 keys per tile
constexpr uint32_t ST_AGG = 1u << 30;           // look-back word: tile's own digit count
constexpr uint32_t ST_INC = 2u << 30;           // look-back word: count of this and all earlier tiles
constexpr uint32_t ST_VAL = (1u << 30) - 1u;
constexpr int OS_SPIN_LIMIT = 1 << 20;

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread over a block of OS_THREADS threads (warp shuffles).
__device__ __forceinline__ uint32_t block_exclusive_scan256(uint32_t x, uint32_t* s_warp /*[OS_WARPS]*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    uint32_t wp = 0;
#pragma unroll
    for (int w = 0; w < OS_WARPS; ++w) wp += (w < warp) ? s_warp[w] : 0u;
    __syncthreads();
    return wp + inc - x;
}

// Digit histograms of every pass over keys[0, n); with `drop`, keys equal to 0xffffffff are left out.
// n_kept gets the number of keys counted.  hist and n_kept start at zero.
__global__ void __launch_bounds__(OS_THREADS) radix_histogram_kernel(const uint32_t* __restrict__ keys,
                                                                     const uint32_t* __restrict__ n_dev, int passes,
                                                                     int drop, uint32_t* __restrict__ hist,
                                                                     uint32_t* __restrict__ n_kept) {
    __shared__ uint32_t s_h[4][256];
    __shared__ uint32_t s_kept;
    for (int i = threadIdx.x; i < 4 * 256; i += OS_THREADS) (&s_h[0][0])[i] = 0;
    if (threadIdx.x == 0) s_kept = 0;
    __syncthreads();
    const uint32_t n = *n_dev;
    uint32_t kept = 0;
    for (uint32_t i = blockIdx.x * OS_THREADS + threadIdx.x; i < n; i += gridDim.x * OS_THREADS) {
        const uint32_t k = __ldg(keys + i);
        if (drop && k == 0xffffffffu) continue;
        ++kept;
        for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(k >> (8 * p)) & 255u], 1u);
    }
    kept = __reduce_add_sync(0xffffffffu, kept);
    if ((threadIdx.x & 31) == 0 && kept) atomicAdd(&s_kept, kept);
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += OS_THREADS) {
        const uint32_t c = (&s_h[0][0])[i];
        if (c) atomicAdd(hist + i, c);
    }
    if (threadIdx.x == 0 && s_kept) atomicAdd(n_kept, s_kept);
}

// One LSD pass.  n = *n_dev keys are read (dropping 0xffffffff keys if `drop`), the kept ones written;
// without vin the values are the input positions.
__global__ void __launch_bounds__(OS_THREADS) radix_onesweep_kernel(const uint32_t* __restrict__ kin,
                                                                    const uint32_t* __restrict__ vin,
                                                                    uint32_t* __restrict__ kout,
                                                                    uint32_t* __restrict__ vout,
                                                                    const uint32_t* __restrict__ n_dev,
                                                                    const uint32_t* __restrict__ n_out, int shift,
                                                                    int drop, const uint32_t* __restrict__ hist,
                                                                    uint32_t* __restrict__ status,
                                                                    uint32_t* __restrict__ ticket,
                                                                    uint32_t* __restrict__ flags) {
    __shared__ uint32_t s_wcnt[OS_WARPS][256];
    __shared__ uint32_t s_lstart[256];    // first staging slot of each digit in this tile
    __shared__ uint32_t s_gdst[256];      // global destination of each digit's first key of this tile
    __shared__ uint32_t s_keys[OS_TILE];
    __shared__ uint32_t s_vals[OS_TILE];
    __shared__ uint32_t s_warp[OS_WARPS];
    __shared__ uint32_t s_tile, s_cnt255;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    for (int i = threadIdx.x; i < OS_WARPS * 256; i += OS_THREADS) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t n = *n_dev;
    const uint64_t base = (uint64_t)tile * OS_TILE;
    if (base >= n) return;   // every tile below this one is in range, so nobody waits for it
    // ---- load and rank: warp w holds keys [base + 32 IPT w, base + 32 IPT (w + 1)), key i of a lane at
    // offset 32 i + lane, ranked in (i, lane) order, i.e. in input order
    const uint32_t lmask = lanemask_lt();
    uint32_t key[OS_IPT], val[OS_IPT], loc[OS_IPT];
#pragma unroll
    for (int i = 0; i < OS_IPT; ++i) {
        const uint64_t g = base + (uint64_t)warp * 32 * OS_IPT + i * 32 + lane;
        bool ok = g < n;
        key[i] = ok ? __ldg(kin + g) : 0xffffffffu;
        val[i] = ok ? (vin ? __ldg(vin + g) : (uint32_t)g) : 0u;
        if (drop && key[i] == 0xffffffffu) ok = false;
        const uint32_t d = (key[i] >> shift) & 255u;
        uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const bool bit = (d >> b) & 1u;
            const uint32_t m = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? m : ~m;
        }
        const int leader = peers ? __ffs(peers) - 1 : lane;
        uint32_t before = 0;
        if (ok && lane == leader) {
            before = s_wcnt[warp][d];
            s_wcnt[warp][d] = before + __popc(peers);
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        loc[i] = ok ? before + __popc(peers & lmask) : 0xffffffffu;
        __syncwarp();
    }
    __syncthreads();
    // ---- per digit: exclusive prefix over warps, the tile's count, then publish it
    const int d = threadIdx.x;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < OS_WARPS; ++w) {
        const uint32_t c = s_wcnt[w][d];
        s_wcnt[w][d] = cnt;
        cnt += c;
    }
    uint32_t* st = status + (uint64_t)tile * 256;
    if (tile == 0) st_relaxed(st + d, ST_INC | cnt);
    else st_relaxed(st + d, ST_AGG | cnt);
    const uint32_t lstart = block_exclusive_scan256(cnt, s_warp);
    s_lstart[d] = lstart;
    // global start of digit d over the whole input (exclusive scan of the pass histogram)
    const uint32_t gstart = block_exclusive_scan256(hist[d], s_warp);
    // ---- decoupled look-back over earlier tiles for digit d
    uint32_t excl = 0;
    for (int64_t j = (int64_t)tile - 1; j >= 0; --j) {
        const uint32_t* p = status + (uint64_t)j * 256 + d;
        uint32_t v = ld_relaxed(p);
        int spins = 0;
        while ((v & (ST_AGG | ST_INC)) == 0 && spins < OS_SPIN_LIMIT) {
            if (++spins > 32) __nanosleep(64);
            v = ld_relaxed(p);
        }
        if ((v & (ST_AGG | ST_INC)) == 0) {   // gave up: the result is wrong, the flag says so
            atomicOr(flags, FLAG_SORT_TIMEOUT);
            break;
        }
        excl += v & ST_VAL;
        if (v & ST_INC) break;
    }
    if (tile > 0) st_relaxed(st + d, ST_INC | (excl + cnt));
    s_gdst[d] = gstart + excl;
    if (d == 255) s_cnt255 = cnt;
    __syncthreads();
    // ---- stage by digit in shared memory, then write runs out
#pragma unroll
    for (int i = 0; i < OS_IPT; ++i) {
        if (loc[i] != 0xffffffffu) {
            const uint32_t dd = (key[i] >> shift) & 255u;
            const uint32_t pos = s_lstart[dd] + s_wcnt[warp][dd] + loc[i];
            s_keys[pos] = key[i];
            s_vals[pos] = val[i];
        }
    }
    __syncthreads();
    const uint32_t kept = s_lstart[255] + s_cnt255;
    const uint32_t n_written = *n_out;   // destinations stay below it even if a look-back gave up
    for (uint32_t j = threadIdx.x; j < kept; j += OS_THREADS) {
        const uint32_t k = s_keys[j];
        const uint32_t dd = (k >> shift) & 255u;
        const uint32_t dst = s_gdst[dd] + (j - s_lstart[dd]);
        if (dst < n_written) {
            kout[dst] = k;
            vout[dst] = s_vals[j];
        }
    }
}

size_t radix_work_words(int64_t n_cap) {
    const int64_t tiles = std::max<int64_t>(1, (n_cap + OS_TILE - 1) / OS_TILE);
    return (size_t)(RADIX_HEADER_WORDS + 4 * tiles * 256);
}

cudaError_t radix_sort_pairs(const uint32_t* kin, const uint32_t* vin, uint32_t* ka, uint32_t* va, uint32_t* kb,
                             uint32_t* vb, const uint32_t* n_dev, int64_t n_cap, int bits, bool drop_max,
                             uint32_t* n_kept, const SortWork& w, bool* result_in_a, cudaStream_t s) {
    *result_in_a = false;
    if (n_cap <= 0) return cudaMemsetAsync(n_kept, 0, sizeof(uint32_t), s);
    if (n_cap >= (1LL << 30) || bits < 1 || bits > 32) return cudaErrorInvalidValue;
    const int passes = (bits + 7) / 8;
    const int64_t tiles = (n_cap + OS_TILE - 1) / OS_TILE;
    if (radix_work_words(n_cap) > w.words) return cudaErrorInvalidValue;
    uint32_t* tickets = w.work;            // [4]
    uint32_t* hist = w.work + 64;          // [4][256]
    uint32_t* status = w.work + RADIX_HEADER_WORDS;
    cudaError_t e = cudaMemsetAsync(w.work, 0, sizeof(uint32_t) * (RADIX_HEADER_WORDS + (size_t)passes * tiles * 256), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_kept, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const unsigned hg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_cap + 4095) / 4096, 4 * (int64_t)w.num_sms));
    radix_histogram_kernel<<<hg, OS_THREADS, 0, s>>>(kin, n_dev, passes, drop_max ? 1 : 0, hist, n_kept);
    // pass p reads (kin, vin) for p = 0, then alternates (ka, va) -> (kb, vb) -> (ka, va) ...
    for (int p = 0; p < passes; ++p) {
        const bool to_a = (p % 2) == 0;
        const uint32_t* ki = p == 0 ? kin : (to_a ? kb : ka);
        const uint32_t* vi = p == 0 ? vin : (to_a ? vb : va);
        radix_onesweep_kernel<<<(unsigned)tiles, OS_THREADS, 0, s>>>(
            ki, vi, to_a ? ka : kb, to_a ? va : vb, p == 0 ? n_dev : n_kept, n_kept, 8 * p, (p == 0 && drop_max) ? 1 : 0,
            hist + 256 * p, status + (size_t)p * tiles * 256, tickets + p, w.flags);
    }
    *result_in_a = (passes % 2) == 1;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ scan

constexpr int SC_BLOCK = 256;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* s_warp, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < SC_BLOCK / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        if (lane < SC_BLOCK / 32) s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t wprefix = warp ? s_warp[warp - 1] : 0u;
    *total = s_warp[SC_BLOCK / 32 - 1];
    __syncthreads();
    return wprefix + inc - x;
}

__device__ __forceinline__ void scan_range(uint32_t n, int G, int b, uint32_t* begin, uint32_t* end) {
    const uint32_t per = ((n + G - 1) / G + SC_BLOCK - 1) / SC_BLOCK * SC_BLOCK;
    const uint64_t b0 = (uint64_t)b * per, b1 = b0 + per;
    *begin = (uint32_t)(b0 < n ? b0 : n);
    *end = (uint32_t)(b1 < n ? b1 : n);
}

__device__ __forceinline__ uint32_t scan_item(const uint32_t* __restrict__ in, const uint32_t* __restrict__ idx,
                                              uint32_t i) {
    return __ldg(in + (idx ? __ldg(idx + i) : i));
}

__global__ void __launch_bounds__(SC_BLOCK) scan_reduce_kernel(const uint32_t* __restrict__ in,
                                                               const uint32_t* __restrict__ idx,
                                                               const uint32_t* __restrict__ n_dev,
                                                               uint32_t* __restrict__ partial) {
    __shared__ uint32_t s_warp[SC_BLOCK / 32];
    uint32_t begin, end;
    scan_range(*n_dev, gridDim.x, blockIdx.x, &begin, &end);
    uint32_t sum = 0;
    for (uint32_t i = begin + threadIdx.x; i < end; i += SC_BLOCK) sum += scan_item(in, idx, i);
    uint32_t total;
    block_exclusive_scan(sum, s_warp, &total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// exclusive scan of the G block partials in place (one block of 1024 threads), total to *total_out
__global__ void __launch_bounds__(1024) scan_partials_kernel(uint32_t* __restrict__ partial, int G,
                                                             uint32_t* __restrict__ total_out) {
    __shared__ uint32_t s_w[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (G + 1023) / 1024;
    const int i0 = threadIdx.x * per, i1 = min(G, i0 + per);
    uint32_t sum = 0;
    for (int i = i0; i < i1; ++i) sum += partial[i];
    uint32_t inc = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t x = s_w[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        s_w[lane] = x;
    }
    __syncthreads();
    uint32_t run = (warp ? s_w[warp - 1] : 0u) + inc - sum;
    for (int i = i0; i < i1; ++i) { const uint32_t x = partial[i]; partial[i] = run; run += x; }
    if (threadIdx.x == 1023) *total_out = s_w[31];
}

__global__ void __launch_bounds__(SC_BLOCK) scan_down_kernel(const uint32_t* __restrict__ in,
                                                             const uint32_t* __restrict__ idx,
                                                             const uint32_t* __restrict__ n_dev,
                                                             const uint32_t* __restrict__ partial,
                                                             uint32_t* __restrict__ out) {
    __shared__ uint32_t s_warp[SC_BLOCK / 32];
    uint32_t begin, end;
    scan_range(*n_dev, gridDim.x, blockIdx.x, &begin, &end);
    uint32_t run = partial[blockIdx.x];
    for (uint32_t i0 = begin; i0 < end; i0 += SC_BLOCK) {
        const uint32_t i = i0 + threadIdx.x;
        const uint32_t x = i < end ? scan_item(in, idx, i) : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(x, s_warp, &total);
        if (i < end) out[i] = run + ex;
        run += total;
    }
}

cudaError_t scan_gathered(const uint32_t* in, const uint32_t* idx, uint32_t* out, const uint32_t* n_dev,
                          uint32_t* total, const SortWork& w, cudaStream_t s) {
    scan_reduce_kernel<<<w.scan_blocks, SC_BLOCK, 0, s>>>(in, idx, n_dev, w.partial);
    scan_partials_kernel<<<1, 1024, 0, s>>>(w.partial, w.scan_blocks, total);
    scan_down_kernel<<<w.scan_blocks, SC_BLOCK, 0, s>>>(in, idx, n_dev, w.partial, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ duplication
//
// Entry i of the depth order (splat m = order[i]) writes its pairs at [pair_off[i], pair_off[i] +
// tiles[m]): key = global tile id, value = m, tiles in row-major order.  A warp takes 32 consecutive
// entries and walks each entry's tiles with all its lanes (a few splats cover thousands of tiles).
__global__ void __launch_bounds__(256) duplicate_kernel(const DevCam* __restrict__ cams, int n_cams,
                                                        const int64_t* __restrict__ cut_offsets, SplatBufs sb,
                                                        const uint32_t* __restrict__ order,
                                                        const uint32_t* __restrict__ n_order,
                                                        const uint32_t* __restrict__ pair_off,
                                                        const uint32_t* __restrict__ n_pairs, int64_t cap_pairs,
                                                        uint32_t* __restrict__ n_pairs_kept,
                                                        uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                        uint32_t* __restrict__ flags) {
    const uint32_t V = *n_order;
    const int lane = threadIdx.x & 31;
    const uint32_t warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t P = *n_pairs;
        *n_pairs_kept = (int64_t)P > cap_pairs ? (uint32_t)cap_pairs : P;
        if ((int64_t)P > cap_pairs) atomicOr(flags, FLAG_PAIRS_OVERFLOW);
    }
    for (uint32_t i0 = warp_global * 32; i0 < V; i0 += n_warps * 32) {
        const uint32_t i = i0 + lane;
        uint32_t nt = 0, rx = 0, ry = 0, m = 0, off = 0;
        int64_t tb = 0;
        int TX = 0;
        if (i < V) {
            m = __ldg(order + i);
            nt = __ldg(sb.tiles + m);
            off = __ldg(pair_off + i);
            if (nt) {
                const uint2 r = sb.rect[m];
                rx = r.x;
                ry = r.y;
                const int k = find_cam(cut_offsets, n_cams, m);
                tb = cams[k].tile_base;
                TX = cams[k].tiles_x;
            }
        }
        uint32_t todo = __ballot_sync(0xffffffffu, nt != 0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint32_t snt = __shfl_sync(0xffffffffu, nt, src);
            const uint32_t srx = __shfl_sync(0xffffffffu, rx, src);
            const uint32_t sry = __shfl_sync(0xffffffffu, ry, src);
            const uint32_t sm = __shfl_sync(0xffffffffu, m, src);
            const uint32_t soff = __shfl_sync(0xffffffffu, off, src);
            const int64_t stb = __shfl_sync(0xffffffffu, tb, src);
            const int sTX = __shfl_sync(0xffffffffu, TX, src);
            const int x0 = srx & 0xffff, x1 = srx >> 16, y0 = sry & 0xffff;
            const uint32_t w = (uint32_t)(x1 - x0 + 1);
            for (uint32_t k = lane; k < snt; k += 32) {
                const uint32_t slot = soff + k;
                if ((int64_t)slot >= cap_pairs) break;
                const uint32_t ty = k / w, tx = k - ty * w;
                keys[slot] = (uint32_t)(stb + (int64_t)(y0 + (int)ty) * sTX + x0 + (int)tx);
                vals[slot] = sm;
            }
        }
    }
}

cudaError_t launch_duplicate(const DevCam* cams, int n_cams, const int64_t* cut_offsets, const SplatBufs& sb,
                             const uint32_t* order, const uint32_t* n_order, const uint32_t* pair_off,
                             const uint32_t* n_pairs, int64_t cap_pairs, uint32_t* n_pairs_kept, uint32_t* keys,
                             uint32_t* vals, uint32_t* flags, int grid, cudaStream_t s) {
    duplicate_kernel<<<grid, 256, 0, s>>>(cams, n_cams, cut_offsets, sb, order, n_order, pair_off, n_pairs, cap_pairs,
                                          n_pairs_kept, keys, vals, flags);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ ranges
//
// ranges[t] = [first, last + 1) of tile id t in the sorted keys (tiles without pairs keep the zero
// range they were cleared to).
__global__ void ranges_kernel(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ n_dev,
                              uint32_t n_tiles, int2* __restrict__ ranges) {
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t k = __ldg(keys + i);
        if (k >= n_tiles) continue;   // only after a failed sort (flagged)
        if (i == 0 || __ldg(keys + i - 1) != k) ranges[k].x = (int)i;
        if (i + 1 == n || __ldg(keys + i + 1) != k) ranges[k].y = (int)(i + 1);
    }
}

cudaError_t launch_ranges(const uint32_t* keys, const uint32_t* n_dev, int64_t n_tiles, int2* ranges, int grid,
                          cudaStream_t s) {
    ranges_kernel<<<grid, 256, 0, s>>>(keys, n_dev, (uint32_t)n_tiles, ranges);
    return cudaGetLastError();
}

}  // namespace h3dgs
