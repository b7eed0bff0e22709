// Binning (a5) and tile ranges (a6): depth sort of the splats, duplication into (tile, splat)
// pairs in depth order, stable sort of the pairs by tile, range detection.
//
// Splats are first sorted by their fp32 depth (4 LSD passes over M splats), then every visible
// splat emits one pair per covered tile in that order, and the pairs are sorted stably by tile id
// (ceil(log2 tiles) bits, 2 passes at 1080p).  Stability keeps every tile's list in (depth, cut
// position) order without sorting 45-bit (tile, depth) keys over all pairs.
//
// The radix sort is a fixed-grid, three-kernel LSD sort with 8-bit digits: per-block digit
// histograms, per-digit scans over blocks, then a scatter that ranks keys stably inside each
// 2048-key tile with warp match/popc, stages them in shared memory by digit and writes runs out
// coalesced.  All element counts live in device memory, so no launch depends on the host.
#include "internal.cuh"

namespace h3dgs {

constexpr int RS_BLOCK = 256;
constexpr int RS_WARPS = RS_BLOCK / 32;
constexpr int RS_IPT = 8;
constexpr int RS_TILE = RS_BLOCK * RS_IPT;

// Per block: [begin, end) of the n keys, in whole tiles, for a grid of G blocks.
__device__ __forceinline__ void block_range(uint32_t n, int G, int b, uint32_t* begin, uint32_t* end) {
    const uint32_t tiles = (n + RS_TILE - 1) / RS_TILE;
    const uint32_t per = (tiles + G - 1) / G;
    const uint64_t b0 = (uint64_t)b * per * RS_TILE;
    const uint64_t b1 = b0 + (uint64_t)per * RS_TILE;
    *begin = (uint32_t)(b0 < n ? b0 : n);
    *end = (uint32_t)(b1 < n ? b1 : n);
}

__global__ void __launch_bounds__(RS_BLOCK) radix_hist_kernel(const uint32_t* __restrict__ keys,
                                                              const uint32_t* __restrict__ n_dev, int shift,
                                                              uint32_t* __restrict__ hist) {
    __shared__ uint32_t s_h[RS_WARPS][256];
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_BLOCK) (&s_h[0][0])[i] = 0;
    __syncthreads();
    uint32_t begin, end;
    block_range(*n_dev, gridDim.x, blockIdx.x, &begin, &end);
    const int warp = threadIdx.x >> 5;
    for (uint32_t i = begin + threadIdx.x; i < end; i += RS_BLOCK)
        atomicAdd(&s_h[warp][(__ldg(keys + i) >> shift) & 255u], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += RS_BLOCK) {
        uint32_t s = 0;
        for (int w = 0; w < RS_WARPS; ++w) s += s_h[w][d];
        hist[(int64_t)d * gridDim.x + blockIdx.x] = s;
    }
}

// One block per digit: exclusive scan of hist[d][0..G) in place, digit total to digit_total[d].
__global__ void radix_scan_kernel(uint32_t* __restrict__ hist, int G, uint32_t* __restrict__ digit_total) {
    __shared__ uint32_t s_part[256];
    uint32_t* h = hist + (int64_t)blockIdx.x * G;
    const int per = (G + blockDim.x - 1) / blockDim.x;
    const int s0 = threadIdx.x * per, s1 = min(G, s0 + per);
    uint32_t sum = 0;
    for (int i = s0; i < s1; ++i) sum += h[i];
    // block exclusive scan of the per-thread sums (blockDim = 256)
    s_part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        uint32_t x = threadIdx.x >= off ? s_part[threadIdx.x - off] : 0u;
        __syncthreads();
        s_part[threadIdx.x] += x;
        __syncthreads();
    }
    uint32_t run = s_part[threadIdx.x] - sum;
    if (threadIdx.x == 255) digit_total[blockIdx.x] = s_part[255];
    for (int i = s0; i < s1; ++i) { const uint32_t x = h[i]; h[i] = run; run += x; }
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__global__ void __launch_bounds__(RS_BLOCK) radix_scatter_kernel(const uint32_t* __restrict__ kin,
                                                                 const uint32_t* __restrict__ vin,
                                                                 uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                                 const uint32_t* __restrict__ n_dev, int shift,
                                                                 const uint32_t* __restrict__ hist,
                                                                 const uint32_t* __restrict__ digit_total) {
    __shared__ uint32_t s_wcnt[RS_WARPS][256];
    __shared__ uint32_t s_tile_cnt[256];
    __shared__ uint32_t s_tile_start[256];
    __shared__ uint32_t s_dst[256];
    __shared__ uint32_t s_keys[RS_TILE];
    __shared__ uint32_t s_vals[RS_TILE];
    __shared__ uint32_t s_scan[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n = *n_dev;
    uint32_t begin, end;
    block_range(n, gridDim.x, blockIdx.x, &begin, &end);
    // global start of each digit for this block = sum of totals of smaller digits + block prefix
    {
        const int d = threadIdx.x;  // RS_BLOCK == 256
        const uint32_t tot = digit_total[d];
        s_scan[d] = tot;
        __syncthreads();
        for (int off = 1; off < 256; off <<= 1) {
            uint32_t x = d >= off ? s_scan[d - off] : 0u;
            __syncthreads();
            s_scan[d] += x;
            __syncthreads();
        }
        s_dst[d] = s_scan[d] - tot + hist[(int64_t)d * gridDim.x + blockIdx.x];
    }
    const uint32_t lmask = lanemask_lt();
    for (uint32_t t0 = begin; t0 < end; t0 += RS_TILE) {
        for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_BLOCK) (&s_wcnt[0][0])[i] = 0;
        __syncthreads();
        uint32_t key[RS_IPT], val[RS_IPT], loc[RS_IPT];
        const uint32_t wbase = t0 + warp * 32 * RS_IPT;
#pragma unroll
        for (int i = 0; i < RS_IPT; ++i) {
            const uint32_t g = wbase + i * 32 + lane;
            const bool ok = g < end;
            key[i] = ok ? __ldg(kin + g) : 0u;
            val[i] = ok ? __ldg(vin + g) : 0u;
            const uint32_t d = ok ? ((key[i] >> shift) & 255u) : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (ok) {
                const int leader = __ffs(peers) - 1;
                uint32_t b = 0;
                if (lane == leader) {
                    b = s_wcnt[warp][d];
                    s_wcnt[warp][d] = b + __popc(peers);
                }
                b = __shfl_sync(peers, b, leader);
                loc[i] = b + __popc(peers & lmask);
            }
            __syncwarp();
        }
        __syncthreads();
        {
            const int d = threadIdx.x;
            uint32_t run = 0;
            for (int w = 0; w < RS_WARPS; ++w) {
                const uint32_t c = s_wcnt[w][d];
                s_wcnt[w][d] = run;
                run += c;
            }
            s_tile_cnt[d] = run;
            s_scan[d] = run;
            __syncthreads();
            for (int off = 1; off < 256; off <<= 1) {
                uint32_t x = d >= off ? s_scan[d - off] : 0u;
                __syncthreads();
                s_scan[d] += x;
                __syncthreads();
            }
            s_tile_start[d] = s_scan[d] - run;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < RS_IPT; ++i) {
            const uint32_t g = wbase + i * 32 + lane;
            if (g < end) {
                const uint32_t d = (key[i] >> shift) & 255u;
                const uint32_t pos = s_tile_start[d] + s_wcnt[warp][d] + loc[i];
                s_keys[pos] = key[i];
                s_vals[pos] = val[i];
            }
        }
        __syncthreads();
        const uint32_t cnt = min((uint32_t)RS_TILE, end - t0);
        for (uint32_t j = threadIdx.x; j < cnt; j += RS_BLOCK) {
            const uint32_t k = s_keys[j];
            const uint32_t d = (k >> shift) & 255u;
            const uint32_t dst = s_dst[d] + (j - s_tile_start[d]);
            kout[dst] = k;
            vout[dst] = s_vals[j];
        }
        __syncthreads();
        s_dst[threadIdx.x] += s_tile_cnt[threadIdx.x];
        __syncthreads();
    }
}

cudaError_t radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const uint32_t* n_dev, int bits,
                             const SortWork& w, bool* result_in_1, cudaStream_t s) {
    bool in1 = false;
    for (int shift = 0; shift < bits; shift += 8) {
        const uint32_t* ki = in1 ? k1 : k0;
        const uint32_t* vi = in1 ? v1 : v0;
        uint32_t* ko = in1 ? k0 : k1;
        uint32_t* vo = in1 ? v0 : v1;
        radix_hist_kernel<<<w.blocks, RS_BLOCK, 0, s>>>(ki, n_dev, shift, w.hist);
        radix_scan_kernel<<<256, 256, 0, s>>>(w.hist, w.blocks, w.digit_total);
        radix_scatter_kernel<<<w.blocks, RS_BLOCK, 0, s>>>(ki, vi, ko, vo, n_dev, shift, w.hist, w.digit_total);
        in1 = !in1;
    }
    *result_in_1 = in1;
    return cudaGetLastError();
}

__global__ void iota_kernel(uint32_t* __restrict__ out, const uint32_t* __restrict__ n_dev) {
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = i;
}

cudaError_t launch_iota(uint32_t* out, const uint32_t* n_dev, int grid, cudaStream_t s) {
    iota_kernel<<<grid, 256, 0, s>>>(out, n_dev);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ gathered scan

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

__global__ void __launch_bounds__(SC_BLOCK) scan_reduce_kernel(const uint32_t* __restrict__ in,
                                                               const uint32_t* __restrict__ idx,
                                                               const uint32_t* __restrict__ n_dev,
                                                               uint32_t* __restrict__ partial) {
    __shared__ uint32_t s_warp[SC_BLOCK / 32];
    uint32_t begin, end;
    scan_range(*n_dev, gridDim.x, blockIdx.x, &begin, &end);
    uint32_t sum = 0;
    for (uint32_t i = begin + threadIdx.x; i < end; i += SC_BLOCK) sum += __ldg(in + __ldg(idx + i));
    uint32_t total;
    block_exclusive_scan(sum, s_warp, &total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// exclusive scan of the G block partials in place (one block of 1024 threads), total to *total_out
__global__ void __launch_bounds__(1024) scan_partials_kernel(uint32_t* __restrict__ partial, int G,
                                                             uint32_t* __restrict__ total_out) {
    __shared__ uint32_t s[1024];
    const int per = (G + 1023) / 1024;
    const int i0 = threadIdx.x * per, i1 = min(G, i0 + per);
    uint32_t sum = 0;
    for (int i = i0; i < i1; ++i) sum += partial[i];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t x = (int)threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += x;
        __syncthreads();
    }
    uint32_t run = s[threadIdx.x] - sum;
    for (int i = i0; i < i1; ++i) { const uint32_t x = partial[i]; partial[i] = run; run += x; }
    if (threadIdx.x == 1023) *total_out = s[1023];
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
        const uint32_t x = i < end ? __ldg(in + __ldg(idx + i)) : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(x, s_warp, &total);
        if (i < end) out[i] = run + ex;
        run += total;
    }
}

cudaError_t scan_gathered(const uint32_t* in, const uint32_t* idx, uint32_t* out, const uint32_t* n_dev,
                          uint32_t* total, const SortWork& w, cudaStream_t s) {
    scan_reduce_kernel<<<w.blocks, SC_BLOCK, 0, s>>>(in, idx, n_dev, w.partial);
    scan_partials_kernel<<<1, 1024, 0, s>>>(w.partial, w.blocks, total);
    scan_down_kernel<<<w.blocks, SC_BLOCK, 0, s>>>(in, idx, n_dev, w.partial, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ duplicate + ranges

// For the splat at depth-sorted position i: one (global tile id, splat) pair per covered tile,
// written from pair_off[i] on, tiles in row-major order.
__global__ void __launch_bounds__(256) duplicate_kernel(const DevCam* __restrict__ cams, int n_cams,
                                                        const int64_t* __restrict__ cut_offsets, SplatBufs sb,
                                                        const uint32_t* __restrict__ order,
                                                        const uint32_t* __restrict__ pair_off,
                                                        const uint32_t* __restrict__ n_pairs, int64_t cap_pairs,
                                                        uint32_t* __restrict__ n_pairs_kept,
                                                        uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                        uint32_t* __restrict__ flags) {
    const uint32_t M = *sb.n_splats;
    const uint32_t P = *n_pairs;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if ((int64_t)P > cap_pairs) atomicOr(flags, FLAG_PAIRS_OVERFLOW);
        *n_pairs_kept = (int64_t)P > cap_pairs ? (uint32_t)cap_pairs : P;
    }
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        const uint32_t m = order[i];
        const uint32_t nt = sb.tiles[m];
        if (nt == 0) continue;
        const uint2 r = sb.rect[m];
        const int x0 = r.x & 0xffff, x1 = r.x >> 16, y0 = r.y & 0xffff, y1 = r.y >> 16;
        const int k = find_cam(cut_offsets, n_cams, m);
        const int64_t tb = cams[k].tile_base;
        const int TX = cams[k].tiles_x;
        int64_t off = pair_off[i];
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x, ++off) {
                if (off < cap_pairs) {
                    keys[off] = (uint32_t)(tb + (int64_t)y * TX + x);
                    vals[off] = m;
                }
            }
    }
}

cudaError_t launch_duplicate(const DevCam* cams, int n_cams, const int64_t* cut_offsets, const SplatBufs& sb,
                             const uint32_t* order, const uint32_t* pair_off, const uint32_t* n_pairs, int64_t cap_pairs,
                             uint32_t* n_pairs_kept, uint32_t* keys, uint32_t* vals, uint32_t* flags, int grid,
                             cudaStream_t s) {
    duplicate_kernel<<<grid, 256, 0, s>>>(cams, n_cams, cut_offsets, sb, order, pair_off, n_pairs, cap_pairs,
                                          n_pairs_kept, keys, vals, flags);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) ranges_kernel(const uint32_t* __restrict__ keys,
                                                     const uint32_t* __restrict__ n_pairs_kept, int2* __restrict__ ranges) {
    const uint32_t P = *n_pairs_kept;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (i == 0 || keys[i - 1] != k) ranges[k].x = (int)i;
        if (i + 1 == P || keys[i + 1] != k) ranges[k].y = (int)(i + 1);
    }
}

cudaError_t launch_ranges(const uint32_t* keys, const uint32_t* n_pairs_kept, int2* ranges, int grid, cudaStream_t s) {
    ranges_kernel<<<grid, 256, 0, s>>>(keys, n_pairs_kept, ranges);
    return cudaGetLastError();
}

}  // namespace h3dgs

namespace h3dgs {

// ------------------------------------------------------------------------------ per-tile depth sort
//
// After the stable sort of the pairs by tile, every tile's entries are in cut-position order.  The
// tile's list is then ordered by (fp32 depth, cut position) with a bitonic network on 64-bit keys
// (depth bits << 32 | cut position; unique) held in shared memory.  Lists are classed by length:
// up to SORT_SMALL entries (16 KB of keys, many CTAs per SM), up to SORT_LARGE (128 KB, one CTA per
// SM), and longer lists sorted in place in a global 64-bit scratch by the same network.

constexpr int SORT_SMALL = 2048;
constexpr int SORT_LARGE = 16384;

__device__ __forceinline__ void bitonic_smem(unsigned long long* s, int N) {
    // N is a power of two <= the block's key capacity; ends with a barrier
    for (int k = 2; k <= N; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int p = threadIdx.x; p < (N >> 1); p += blockDim.x) {
                const int pos = 2 * j * (p / j) + (p % j);
                const int q = pos + j;
                const bool up = (pos & k) == 0;
                const unsigned long long a = s[pos], b = s[q];
                if ((a > b) == up) { s[pos] = b; s[q] = a; }
            }
            __syncthreads();
        }
}

// Sorts one tile's list [r.x, r.y) in shared memory (n <= CAP entries).
__device__ __forceinline__ void sort_tile_smem(unsigned long long* s_key, int2 r, const uint32_t* __restrict__ depth_key,
                                               uint32_t* __restrict__ list) {
    const int n = r.y - r.x;
    int N = 1;
    while (N < n) N <<= 1;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        if (i < n) {
            const uint32_t m = list[r.x + i];
            s_key[i] = ((unsigned long long)__ldg(depth_key + m) << 32) | m;
        } else {
            s_key[i] = ~0ull;
        }
    }
    __syncthreads();
    bitonic_smem(s_key, N);
    for (int i = threadIdx.x; i < n; i += blockDim.x) list[r.x + i] = (uint32_t)(s_key[i] & 0xffffffffu);
    __syncthreads();
}

// lists of 2 .. SORT_SMALL entries: one CTA per tile; longer lists are appended to the large/huge
// work lists for the persistent kernels below
__global__ void __launch_bounds__(256) tile_sort_small_kernel(const int2* __restrict__ ranges, int64_t n_tiles,
                                                              const uint32_t* __restrict__ depth_key,
                                                              uint32_t* __restrict__ list, uint32_t* __restrict__ large,
                                                              uint32_t* __restrict__ n_large, uint32_t* __restrict__ huge,
                                                              uint32_t* __restrict__ n_huge) {
    __shared__ unsigned long long s_key[SORT_SMALL];
    const int64_t tile = blockIdx.x;
    if (tile >= n_tiles) return;
    const int2 r = ranges[tile];
    const int n = r.y - r.x;
    if (n < 2) return;
    if (n > SORT_SMALL) {
        if (threadIdx.x == 0) {
            if (n > SORT_LARGE) huge[atomicAdd(n_huge, 1u)] = (uint32_t)tile;
            else large[atomicAdd(n_large, 1u)] = (uint32_t)tile;
        }
        return;
    }
    sort_tile_smem(s_key, r, depth_key, list);
}

// lists of SORT_SMALL .. SORT_LARGE entries: persistent CTAs of 1024 threads with 128 KB of keys
__global__ void __launch_bounds__(1024) tile_sort_large_kernel(const int2* __restrict__ ranges,
                                                               const uint32_t* __restrict__ depth_key,
                                                               uint32_t* __restrict__ list,
                                                               const uint32_t* __restrict__ large,
                                                               const uint32_t* __restrict__ n_large) {
    extern __shared__ unsigned long long s_key[];
    const uint32_t cnt = *n_large;
    for (uint32_t i = blockIdx.x; i < cnt; i += gridDim.x) sort_tile_smem(s_key, ranges[large[i]], depth_key, list);
}

// lists longer than SORT_LARGE: the same network over a global 64-bit scratch (rare)
__global__ void __launch_bounds__(1024) tile_sort_huge_kernel(const int2* __restrict__ ranges,
                                                              const uint32_t* __restrict__ depth_key,
                                                              uint32_t* __restrict__ list,
                                                              const uint32_t* __restrict__ huge,
                                                              const uint32_t* __restrict__ n_huge,
                                                              unsigned long long* __restrict__ scratch,
                                                              int64_t scratch_cap) {
    const uint32_t cnt = *n_huge;
    for (uint32_t ti = blockIdx.x; ti < cnt; ti += gridDim.x) {
        const int2 r = ranges[huge[ti]];
        const int n = r.y - r.x;
        int N = 1;
        while (N < n) N <<= 1;
        // the tile's padded segment lives at [2 r.x, 2 r.x + N) of the scratch (N < 2n: disjoint)
        const int64_t base = 2 * (int64_t)r.x;
        if (base + N > scratch_cap) continue;
        unsigned long long* s = scratch + base;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            if (i < n) {
                const uint32_t m = list[r.x + i];
                s[i] = ((unsigned long long)__ldg(depth_key + m) << 32) | m;
            } else {
                s[i] = ~0ull;
            }
        }
        __syncthreads();
        for (int k = 2; k <= N; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int p = threadIdx.x; p < (N >> 1); p += blockDim.x) {
                    const int pos = 2 * j * (p / j) + (p % j);
                    const int q = pos + j;
                    const bool up = (pos & k) == 0;
                    const unsigned long long a = s[pos], b = s[q];
                    if ((a > b) == up) { s[pos] = b; s[q] = a; }
                }
                __syncthreads();
            }
        for (int i = threadIdx.x; i < n; i += blockDim.x) list[r.x + i] = (uint32_t)(s[i] & 0xffffffffu);
        __syncthreads();
    }
}

cudaError_t launch_tile_depth_sort(const int2* ranges, int64_t n_tiles, const uint32_t* depth_key, uint32_t* list,
                                   uint32_t* work /*2 n_tiles + 2*/, unsigned long long* scratch, int64_t scratch_cap,
                                   int num_sms, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tile_sort_large_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SORT_LARGE * 8);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    uint32_t* n_large = work;
    uint32_t* n_huge = work + 1;
    uint32_t* large = work + 2;
    uint32_t* huge = work + 2 + n_tiles;
    cudaError_t e = cudaMemsetAsync(work, 0, 2 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    tile_sort_small_kernel<<<(unsigned)n_tiles, 256, 0, s>>>(ranges, n_tiles, depth_key, list, large, n_large, huge, n_huge);
    tile_sort_large_kernel<<<num_sms, 1024, SORT_LARGE * 8, s>>>(ranges, depth_key, list, large, n_large);
    tile_sort_huge_kernel<<<16, 1024, 0, s>>>(ranges, depth_key, list, huge, n_huge, scratch, scratch_cap);
    return cudaGetLastError();
}

// plain exclusive scan of in[0, n) (no gather): out, *total
__global__ void __launch_bounds__(SC_BLOCK) scan_reduce_plain_kernel(const uint32_t* __restrict__ in,
                                                                     const uint32_t* __restrict__ n_dev,
                                                                     uint32_t* __restrict__ partial) {
    __shared__ uint32_t s_warp[SC_BLOCK / 32];
    uint32_t begin, end;
    scan_range(*n_dev, gridDim.x, blockIdx.x, &begin, &end);
    uint32_t sum = 0;
    for (uint32_t i = begin + threadIdx.x; i < end; i += SC_BLOCK) sum += __ldg(in + i);
    uint32_t total;
    block_exclusive_scan(sum, s_warp, &total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SC_BLOCK) scan_down_plain_kernel(const uint32_t* __restrict__ in,
                                                                   const uint32_t* __restrict__ n_dev,
                                                                   const uint32_t* __restrict__ partial,
                                                                   uint32_t* __restrict__ out) {
    __shared__ uint32_t s_warp[SC_BLOCK / 32];
    uint32_t begin, end;
    scan_range(*n_dev, gridDim.x, blockIdx.x, &begin, &end);
    uint32_t run = partial[blockIdx.x];
    for (uint32_t i0 = begin; i0 < end; i0 += SC_BLOCK) {
        const uint32_t i = i0 + threadIdx.x;
        const uint32_t x = i < end ? __ldg(in + i) : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(x, s_warp, &total);
        if (i < end) out[i] = run + ex;
        run += total;
    }
}

cudaError_t scan_plain(const uint32_t* in, uint32_t* out, const uint32_t* n_dev, uint32_t* total, const SortWork& w,
                       cudaStream_t s) {
    scan_reduce_plain_kernel<<<w.blocks, SC_BLOCK, 0, s>>>(in, n_dev, w.partial);
    scan_partials_kernel<<<1, 1024, 0, s>>>(w.partial, w.blocks, total);
    scan_down_plain_kernel<<<w.blocks, SC_BLOCK, 0, s>>>(in, n_dev, w.partial, out);
    return cudaGetLastError();
}

// Pairs in cut order: for splat m, one (global tile id, m) pair per covered tile (row-major).
__global__ void __launch_bounds__(256) duplicate_plain_kernel(const DevCam* __restrict__ cams, int n_cams,
                                                              const int64_t* __restrict__ cut_offsets, SplatBufs sb,
                                                              const uint32_t* __restrict__ pair_off,
                                                              const uint32_t* __restrict__ n_pairs, int64_t cap_pairs,
                                                              uint32_t* __restrict__ n_pairs_kept,
                                                              uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                              uint32_t* __restrict__ flags) {
    const uint32_t M = *sb.n_splats;
    const uint32_t P = *n_pairs;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if ((int64_t)P > cap_pairs) atomicOr(flags, FLAG_PAIRS_OVERFLOW);
        *n_pairs_kept = (int64_t)P > cap_pairs ? (uint32_t)cap_pairs : P;
    }
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const uint32_t nt = sb.tiles[m];
        if (nt == 0) continue;
        const uint2 r = sb.rect[m];
        const int x0 = r.x & 0xffff, x1 = r.x >> 16, y0 = r.y & 0xffff, y1 = r.y >> 16;
        const int k = find_cam(cut_offsets, n_cams, m);
        const int64_t tb = cams[k].tile_base;
        const int TX = cams[k].tiles_x;
        int64_t off = pair_off[m];
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x, ++off) {
                if (off < cap_pairs) {
                    keys[off] = (uint32_t)(tb + (int64_t)y * TX + x);
                    vals[off] = m;
                }
            }
    }
}

cudaError_t launch_duplicate_plain(const DevCam* cams, int n_cams, const int64_t* cut_offsets, const SplatBufs& sb,
                                   const uint32_t* pair_off, const uint32_t* n_pairs, int64_t cap_pairs,
                                   uint32_t* n_pairs_kept, uint32_t* keys, uint32_t* vals, uint32_t* flags, int grid,
                                   cudaStream_t s) {
    duplicate_plain_kernel<<<grid, 256, 0, s>>>(cams, n_cams, cut_offsets, sb, pair_off, n_pairs, cap_pairs, n_pairs_kept,
                                                keys, vals, flags);
    return cudaGetLastError();
}

}  // namespace h3dgs
