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
//   5. tile ranges are marked by the last pass of that sort (the first and last position of each run
//      of equal tile ids in its staging).
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
#include "lookback.cuh"

namespace h3dgs {

// ------------------------------------------------------------------------------ radix sort

constexpr int OS_THREADS = 256;                 // one thread per digit in the look-back
constexpr int OS_WARPS = OS_THREADS / 32;
constexpr int OS_IPT_SMALL = 7;                 // keys per thread when all tiles fit one wave (6..8 measured)
constexpr int OS_IPT_LARGE = 12;                // keys per thread otherwise (10..15 measured)
constexpr int OS_TILE_SMALL = OS_THREADS * OS_IPT_SMALL;   // 1792 keys per tile
constexpr int OS_TILE_LARGE = OS_THREADS * OS_IPT_LARGE;   // 3072 keys per tile
constexpr unsigned long long ST_AGG = 1ull << 62;   // look-back word: tile's own digit count
constexpr unsigned long long ST_INC = 2ull << 62;   // look-back word: count of this and all earlier tiles
constexpr unsigned long long ST_VAL = (1ull << 62) - 1;
constexpr int OS_SPIN_LIMIT = 1 << 20;       // re-reads of one look-back word before giving up
constexpr int OS_LOOKBACK = 8;               // look-back words loaded per step
constexpr int OS_GROUP = 16;                 // tiles per group of the grouped prefix (one-wave passes)
constexpr int HG_IPT = 4;                    // keys per thread of the histogram kernel

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
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
// n_kept gets the number of keys counted.  hist and n_kept start at zero.  Lanes of a warp holding the
// same digit are grouped (8 ballots) and their leader adds the group's size, so skewed digits (the
// top byte of depth keys takes a handful of values) cost one shared atomic per group.
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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lmask = lanemask_lt();
    uint32_t kept = 0;
    // HG_IPT keys per thread, all loads issued before any ranking; a warp covers 32 HG_IPT
    // consecutive keys (whole warps iterate together: the ballots need every lane)
    for (uint64_t w0 = ((uint64_t)blockIdx.x * OS_WARPS + warp) * 32 * HG_IPT; w0 < n;
         w0 += (uint64_t)gridDim.x * OS_WARPS * 32 * HG_IPT) {
        uint32_t kk[HG_IPT];
#pragma unroll
        for (int q = 0; q < HG_IPT; ++q) {
            const uint64_t i = w0 + q * 32 + lane;
            kk[q] = i < n ? __ldg(keys + i) : 0xffffffffu;
        }
#pragma unroll
        for (int q = 0; q < HG_IPT; ++q) {
            const uint64_t i = w0 + q * 32 + lane;
            const uint32_t k = kk[q];
            const bool ok = i < n && !(drop && k == 0xffffffffu);
            kept += ok;
            const uint32_t valid = __ballot_sync(0xffffffffu, ok);
            for (int p = 0; p < passes; ++p) {
                const uint32_t d = (k >> (8 * p)) & 255u;
                uint32_t peers = valid;
#pragma unroll
                for (int bit = 0; bit < 8; ++bit) {
                    const bool on = (d >> bit) & 1u;
                    const uint32_t m = __ballot_sync(0xffffffffu, on);
                    peers &= on ? m : ~m;
                }
                if (ok && (peers & lmask) == 0) atomicAdd(&s_h[p][d], (uint32_t)__popc(peers));
            }
        }
    }
    kept = __reduce_add_sync(0xffffffffu, kept);
    if (lane == 0 && kept) atomicAdd(&s_kept, kept);
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += OS_THREADS) {
        const uint32_t c = (&s_h[0][0])[i];
        if (c) atomicAdd(hist + i, c);
    }
    if (threadIdx.x == 0 && s_kept) atomicAdd(n_kept, s_kept);
}

// One LSD pass.  n = *n_dev keys are read (dropping 0xffffffff keys if `drop`), the kept ones written;
// without vin the values are the input positions.
template <int OS_IPT>
__global__ void __launch_bounds__(OS_THREADS, 3) radix_onesweep_kernel(const uint32_t* __restrict__ kin,
                                                                    const uint32_t* __restrict__ vin,
                                                                    uint32_t* __restrict__ kout,
                                                                    uint32_t* __restrict__ vout,
                                                                    const uint32_t* __restrict__ n_dev,
                                                                    const uint32_t* __restrict__ n_out, int shift,
                                                                    int drop, const uint32_t* __restrict__ hist,
                                                                    unsigned long long* __restrict__ status,
                                                                    uint32_t* __restrict__ gtot,
                                                                    uint32_t* __restrict__ gcnt,
                                                                    uint32_t* __restrict__ ticket,
                                                                    uint32_t* __restrict__ flags,
                                                                    uint32_t* __restrict__ ranges,
                                                                    uint32_t n_ranges) {
    __shared__ uint32_t s_wcnt[OS_WARPS][256];
    __shared__ uint32_t s_lstart[256];    // first staging slot of each digit in this tile
    __shared__ uint32_t s_gdst[256];      // global destination of each digit's first key of this tile
    constexpr int OS_TILE = OS_THREADS * OS_IPT;
    __shared__ uint32_t s_keys[OS_TILE];
    __shared__ uint32_t s_vals[OS_TILE];
    __shared__ uint32_t s_warp[OS_WARPS];
    __shared__ uint32_t s_tile, s_cnt255;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    griddep_launch_dependents();
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);   // tickets are cleared before the frame
    for (int i = threadIdx.x; i < OS_WARPS * 256; i += OS_THREADS) (&s_wcnt[0][0])[i] = 0;
    griddep_wait();
    // loads that do not depend on the tile overlap the ticket
    const uint32_t n = *n_dev;
    const uint32_t n_written = *n_out;   // destinations stay below it even if a look-back gave up
    const uint32_t hist_d = hist[threadIdx.x];
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t base = (uint64_t)tile * OS_TILE;
    if (base >= n) return;   // every tile below this one is in range, so nobody waits for it
    // ---- load and rank: warp w holds keys [base + 32 IPT w, base + 32 IPT (w + 1)), key i of a lane at
    // offset 32 i + lane, ranked in (i, lane) order, i.e. in input order.  All loads are issued first.
    const uint32_t lmask = lanemask_lt();
    uint32_t key[OS_IPT], val[OS_IPT], loc[OS_IPT];
#pragma unroll
    for (int i = 0; i < OS_IPT; ++i) {
        const uint64_t g = base + (uint64_t)warp * 32 * OS_IPT + i * 32 + lane;
        const bool ok = g < n;
        key[i] = ok ? __ldg(kin + g) : 0xffffffffu;
        val[i] = ok ? (vin ? __ldg(vin + g) : (uint32_t)g) : 0u;
    }
#pragma unroll
    for (int i = 0; i < OS_IPT; ++i) {
        const uint64_t g = base + (uint64_t)warp * 32 * OS_IPT + i * 32 + lane;
        bool ok = g < n;
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
    unsigned long long* st = status + (uint64_t)tile * 256;
    if (tile == 0) st_relaxed(st + d, ST_INC | cnt);
    else st_relaxed(st + d, ST_AGG | cnt);
    const uint32_t grp = tile / OS_GROUP;
    if (gcnt) {   // grouped prefix: this tile's share of its group's digit totals
        if (cnt) atomicAdd(gtot + (size_t)grp * 256 + d, cnt);
        __threadfence();
    }
    const uint32_t lstart = block_exclusive_scan256(cnt, s_warp);   // (its barriers order the shares)
    s_lstart[d] = lstart;
    // global start of digit d over the whole input (exclusive scan of the pass histogram)
    const uint32_t gstart = block_exclusive_scan256(hist_d, s_warp);
    unsigned long long excl = 0;
    if (gcnt) {
        // ---- grouped prefix (every tile of the pass is resident, so all earlier tiles publish at about
        // the same time): the digit totals of the complete earlier groups, then the counts of the
        // earlier tiles of this group; all loads are independent, the waits are bounded
        if (threadIdx.x == 0) atomicAdd(gcnt + grp, 1u);   // every share of this tile is in place
        for (uint32_t g = threadIdx.x; g < grp; g += OS_THREADS) {
            int spins = 0;
            while (ld_acquire32(gcnt + g) < (uint32_t)OS_GROUP && spins < OS_SPIN_LIMIT)
                if (++spins > 32) __nanosleep(64);
            if (spins >= OS_SPIN_LIMIT) atomicOr(flags, FLAG_WAIT_TIMEOUT);   // result wrong, flagged
        }
        __syncthreads();
        for (uint32_t g0 = 0; g0 < grp; g0 += 8) {
            uint32_t v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = g0 + q < grp ? ld_relaxed32(gtot + (size_t)(g0 + q) * 256 + d) : 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q) excl += v[q];
        }
        const uint32_t j0 = grp * OS_GROUP;
        unsigned long long v[OS_GROUP - 1];
#pragma unroll
        for (int q = 0; q < OS_GROUP - 1; ++q) v[q] = j0 + q < tile ? ld_relaxed(status + (uint64_t)(j0 + q) * 256 + d) : 0u;
#pragma unroll
        for (int q = 0; q < OS_GROUP - 1; ++q) {
            if (j0 + q >= tile) continue;
            unsigned long long x = v[q];
            int spins = 0;
            while ((x & (ST_AGG | ST_INC)) == 0 && spins < OS_SPIN_LIMIT) {
                if (++spins > 32) __nanosleep(64);
                x = ld_relaxed(status + (uint64_t)(j0 + q) * 256 + d);
            }
            if ((x & (ST_AGG | ST_INC)) == 0) atomicOr(flags, FLAG_WAIT_TIMEOUT);
            else excl += x & ST_VAL;
        }
    } else {
        // ---- decoupled look-back over earlier tiles for digit d: OS_LOOKBACK status words are loaded
        // at once, then summed newest first until an inclusive one; a word not yet published is re-read
        bool found = false;
        for (int64_t j = (int64_t)tile - 1; j >= 0 && !found; j -= OS_LOOKBACK) {
            unsigned long long v[OS_LOOKBACK];
#pragma unroll
            for (int q = 0; q < OS_LOOKBACK; ++q)
                v[q] = (j - q >= 0) ? ld_relaxed(status + (uint64_t)(j - q) * 256 + d) : 0u;
#pragma unroll
            for (int q = 0; q < OS_LOOKBACK; ++q) {
                if (found || j - q < 0) {
                    found = true;
                    continue;
                }
                unsigned long long x = v[q];
                int spins = 0;
                while ((x & (ST_AGG | ST_INC)) == 0 && spins < OS_SPIN_LIMIT) {
                    if (++spins > 32) __nanosleep(64);
                    x = ld_relaxed(status + (uint64_t)(j - q) * 256 + d);
                }
                if ((x & (ST_AGG | ST_INC)) == 0) {   // gave up: the result is wrong, the flag says so
                    atomicOr(flags, FLAG_WAIT_TIMEOUT);
                    found = true;
                    continue;
                }
                excl += x & ST_VAL;
                if (x & ST_INC) found = true;
            }
        }
        if (tile > 0) st_relaxed(st + d, ST_INC | (excl + cnt));
    }
    s_gdst[d] = (uint32_t)(gstart + excl);
    if (d == 255) s_cnt255 = cnt;
    __syncthreads();
    // ---- stage by digit in shared memory, then write runs out
#pragma unroll
    for (int i = 0; i < OS_IPT; ++i) {
        if (loc[i] != 0xffffffffu) {
            const uint32_t dd = (key[i] >> shift) & 255u;
            const uint32_t pos = s_lstart[dd] + s_wcnt[warp][dd] + loc[i];
            if (H3DGS_IN(pos, OS_TILE)) {
                s_keys[pos] = key[i];
                s_vals[pos] = val[i];
            }
        }
    }
    __syncthreads();
    const uint32_t kept = s_lstart[255] + s_cnt255;
    for (uint32_t j = threadIdx.x; j < kept; j += OS_THREADS) {
        const uint32_t k = s_keys[j];
        const uint32_t dd = (k >> shift) & 255u;
        const uint32_t dst = s_gdst[dd] + (j - s_lstart[dd]);
        if (H3DGS_IN(dst, n_written) && dst < n_written) {
            kout[dst] = k;
            vout[dst] = s_vals[j];
            // the last pass of a sort whose keys were already ordered on the lower digits: equal keys
            // are neighbours in the staging, so the first and last of every run mark the key's range
            // (first stored inverted, so that zero means untouched; see radix_sort_pairs)
            if (ranges && k < n_ranges) {
                if (j == 0 || s_keys[j - 1] != k) atomicMax(ranges + 2 * (size_t)k, ~dst);
                if (j + 1 == kept || s_keys[j + 1] != k) atomicMax(ranges + 2 * (size_t)k + 1, dst + 1);
            }
        }
    }
}

// Workspace: header, the 64-bit look-back words [4 passes][tiles][256], then for the grouped prefix
// [4 passes][groups][256] digit totals and [4 passes][groups] completion counters.
static int64_t radix_max_tiles(int64_t n_cap) {
    return std::max<int64_t>(1, (n_cap + OS_TILE_SMALL - 1) / OS_TILE_SMALL);
}
size_t radix_work_words(int64_t n_cap) {
    const int64_t tiles = radix_max_tiles(n_cap), groups = (tiles + OS_GROUP - 1) / OS_GROUP;
    return (size_t)(RADIX_HEADER_WORDS + 2 * 4 * tiles * 256 + 4 * groups * 257);
}

__global__ void reset_kernel(ResetList r) {
    griddep_launch_dependents();
    griddep_wait();
    if (r.cams && blockIdx.x == 0 && (int)threadIdx.x < r.cb.count) setup_camera(r.cb, threadIdx.x, r.cams);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x, t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (int k = 0; k < r.n; ++k) {
        uint32_t* p = r.p[k];
        const uint64_t n = r.words[k];
        if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {   // 16-byte stores, then the tail
            uint4* q = reinterpret_cast<uint4*>(p);
            for (uint64_t i = t0; i < n / 4; i += stride) q[i] = make_uint4(0u, 0u, 0u, 0u);
            for (uint64_t i = (n / 4) * 4 + t0; i < n; i += stride) p[i] = 0u;
        } else {
            for (uint64_t i = t0; i < n; i += stride) p[i] = 0u;
        }
    }
}

cudaError_t launch_reset(const ResetList& r, int num_sms, cudaStream_t s) {
    if (r.n < 0 || r.n > 8) return cudaErrorInvalidValue;
    const cudaError_t e = launch_dependent(reset_kernel, dim3(num_sms * 4), dim3(256), s, r);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t radix_sort_pairs(const uint32_t* kin, const uint32_t* vin, uint32_t* ka, uint32_t* va, uint32_t* kb,
                             uint32_t* vb, const uint32_t* n_dev, int64_t n_cap, int bits, bool drop_max,
                             uint32_t* n_kept, const SortWork& w, bool* result_in_a, cudaStream_t s,
                             const uint32_t* hist_pre, bool pre_zeroed, uint32_t* ranges, int64_t n_ranges) {
    *result_in_a = false;
    if (n_cap <= 0) return hist_pre ? cudaSuccess : cudaMemsetAsync(n_kept, 0, sizeof(uint32_t), s);
    if (n_cap > 0xffffffffLL || bits < 1 || bits > 32) return cudaErrorInvalidValue;
    const int passes = (bits + 7) / 8;
    // small tiles (a shorter serial ranking chain per tile) while every tile of a pass fits one wave of
    // resident blocks, larger tiles beyond
    const bool small = (n_cap + OS_TILE_SMALL - 1) / OS_TILE_SMALL <= 3 * (int64_t)w.num_sms;
    const int64_t tile_keys = small ? OS_TILE_SMALL : OS_TILE_LARGE;
    const int64_t tiles = (n_cap + tile_keys - 1) / tile_keys;
    if (radix_work_words(n_cap) > w.words) return cudaErrorInvalidValue;
    uint32_t* tickets = w.work;            // [4]
    uint32_t* hist = w.work + 64;          // [4][256]
    unsigned long long* status = reinterpret_cast<unsigned long long*>(w.work + RADIX_HEADER_WORDS);
    // grouped prefix when the tiles of a pass are (about) all resident at once: 3 blocks of 256 per SM
    // hold 3 x SMs tiles, and tiles beyond the keys actually present exit at once (the launch is
    // sized by the capacity)
    const int64_t max_tiles = radix_max_tiles(n_cap), max_groups = (max_tiles + OS_GROUP - 1) / OS_GROUP;
    const bool grouped = tiles <= 4 * (int64_t)w.num_sms;
    uint32_t* gtot = w.work + RADIX_HEADER_WORDS + 2 * 4 * max_tiles * 256;   // [4][max_groups][256]
    uint32_t* gcnt = gtot + 4 * max_groups * 256;                             // [4][max_groups]
    cudaError_t e = cudaSuccess;
    if (!pre_zeroed)
        e = cudaMemsetAsync(w.work, 0, sizeof(uint32_t) * RADIX_HEADER_WORDS +
                                           sizeof(unsigned long long) * (size_t)passes * tiles * 256, s);
    if (e == cudaSuccess && !pre_zeroed && grouped) e = cudaMemsetAsync(gtot, 0, sizeof(uint32_t) * 4 * max_groups * 257, s);
    if (e != cudaSuccess) return e;
    if (hist_pre) {
        hist = const_cast<uint32_t*>(hist_pre);   // counted by the producer of the keys, with *n_kept
    } else {
        e = cudaMemsetAsync(n_kept, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
        const int64_t per_block = (int64_t)OS_THREADS * HG_IPT;
        const unsigned hg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_cap + per_block - 1) / per_block,
                                                                             16 * (int64_t)w.num_sms));
        radix_histogram_kernel<<<hg, OS_THREADS, 0, s>>>(kin, n_dev, passes, drop_max ? 1 : 0, hist, n_kept);
    }
    // pass p reads (kin, vin) for p = 0, then alternates (ka, va) -> (kb, vb) -> (ka, va) ...
    for (int p = 0; p < passes; ++p) {
        const bool to_a = (p % 2) == 0;
        const uint32_t* ki = p == 0 ? kin : (to_a ? kb : ka);
        const uint32_t* vi = p == 0 ? vin : (to_a ? vb : va);
        e = launch_dependent(small ? radix_onesweep_kernel<OS_IPT_SMALL> : radix_onesweep_kernel<OS_IPT_LARGE>,
                             dim3((unsigned)tiles), dim3(OS_THREADS), s, ki, vi, to_a ? ka : kb, to_a ? va : vb,
                             p == 0 ? n_dev : n_kept, n_kept, 8 * p, (p == 0 && drop_max) ? 1 : 0, hist + 256 * p,
                             status + (size_t)p * tiles * 256, grouped ? gtot + (size_t)p * max_groups * 256 : nullptr,
                             grouped ? gcnt + (size_t)p * max_groups : nullptr, tickets + p, w.flags,
                             p + 1 == passes ? ranges : nullptr, (uint32_t)std::min<int64_t>(n_ranges, 0xffffffffLL));
        if (e != cudaSuccess) return e;
    }
    *result_in_a = (passes % 2) == 1;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ pair offsets
//
// One pass over the depth order: entry i (splat order[i]) gets its first pair slot pair_off[i] =
// sum of the tile counts of the entries before it (single-pass scan with decoupled look-back), and
// every segment of DUP_SEG pairs records the entry holding its first pair (seg_start), which is
// what the duplication uses to balance pairs over blocks.

constexpr int PO_THREADS = 256;
constexpr int PO_IPT = 8;
constexpr int PO_TILE = PO_THREADS * PO_IPT;

__global__ void __launch_bounds__(PO_THREADS) pair_offsets_kernel(const uint32_t* __restrict__ tiles,
                                                                  const uint32_t* __restrict__ order,
                                                                  const uint32_t* __restrict__ n_dev,
                                                                  uint32_t* __restrict__ pair_off,
                                                                  uint32_t* __restrict__ seg_start, uint32_t seg_cap,
                                                                  uint32_t* __restrict__ total, Lookback lb) {
    griddep_launch_dependents();
    griddep_wait();
    __shared__ uint32_t s_ticket;
    __shared__ unsigned long long s_slot, s_warp[PO_THREADS / 32];
    const uint32_t b = lb_ticket(lb, &s_ticket);
    const uint32_t n = *n_dev;
    const uint64_t base = (uint64_t)b * PO_TILE;
    if (base >= n && b > 0) return;   // block 0 always runs, so that an empty input still gets total = 0
    // thread t owns entries base + t IPT + q, q < IPT (contiguous, so its running sum is in order)
    uint32_t x[PO_IPT];
    unsigned long long sum = 0;
#pragma unroll
    for (int q = 0; q < PO_IPT; ++q) {
        const uint64_t i = base + (uint64_t)threadIdx.x * PO_IPT + q;
        x[q] = i < n ? __ldg(tiles + __ldg(order + i)) : 0u;
        sum += x[q];
    }
    unsigned long long agg;
    const unsigned long long before = lb_block_scan<PO_THREADS>(sum, s_warp, &agg);
    const unsigned long long prefix = lb_prefix(lb, b, agg, &s_slot);
    unsigned long long off = prefix + before;
#pragma unroll
    for (int q = 0; q < PO_IPT; ++q) {
        const uint64_t i = base + (uint64_t)threadIdx.x * PO_IPT + q;
        if (i < n) {
            pair_off[i] = (uint32_t)off;
            if (x[q]) {   // segments whose first pair lies in [off, off + x)
                const uint64_t s0 = (off + DUP_SEG - 1) / DUP_SEG, s1 = (off + x[q] - 1) / DUP_SEG;
                for (uint64_t sg = s0; sg <= s1 && sg < seg_cap; ++sg) seg_start[sg] = (uint32_t)i;
            }
            if (i + 1 == n) *total = (uint32_t)min(off + x[q], (unsigned long long)0xffffffffu);
        }
        off += x[q];
    }
    if (n == 0 && threadIdx.x == 0) *total = 0;
}

size_t pair_offsets_work_words(int64_t n_cap) {
    return LB_HEADER_WORDS + lb_body_words(std::max<int64_t>(1, (n_cap + PO_TILE - 1) / PO_TILE));
}

cudaError_t launch_pair_offsets(const uint32_t* tiles, const uint32_t* order, const uint32_t* n_dev, int64_t n_cap,
                                uint32_t* pair_off, uint32_t* seg_start, int64_t seg_cap, uint32_t* total,
                                const SortWork& w, cudaStream_t s, bool pre_zeroed) {
    const int64_t blocks = std::max<int64_t>(1, (n_cap + PO_TILE - 1) / PO_TILE);
    const size_t words = LB_HEADER_WORDS + lb_body_words(blocks);
    if (words > w.words) return cudaErrorInvalidValue;
    // grouped prefix when every block is resident (a few blocks of 256 per SM)
    const Lookback lb = lb_make(w.work, blocks, blocks <= 4 * (int64_t)w.num_sms, w.flags);
    if (!pre_zeroed) {
        cudaError_t e = cudaMemsetAsync(w.work, 0, sizeof(uint32_t) * words, s);
        if (e != cudaSuccess) return e;
    }
    const cudaError_t e = launch_dependent(pair_offsets_kernel, dim3((unsigned)blocks), dim3(PO_THREADS), s, tiles, order,
                                           n_dev, pair_off, seg_start,
                                           (uint32_t)std::min<int64_t>(seg_cap, 0xffffffffLL), total, lb);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// seg_start from finished pair offsets (used when the segment array had to grow after the scan)
__global__ void pair_segments_kernel(const uint32_t* __restrict__ tiles, const uint32_t* __restrict__ order,
                                     const uint32_t* __restrict__ n_dev, const uint32_t* __restrict__ pair_off,
                                     uint32_t* __restrict__ seg_start, uint32_t seg_cap) {
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t off = __ldg(pair_off + i), x = __ldg(tiles + __ldg(order + i));
        if (!x) continue;
        const uint64_t s0 = (off + DUP_SEG - 1) / DUP_SEG, s1 = (off + x - 1) / DUP_SEG;
        for (uint64_t sg = s0; sg <= s1 && sg < seg_cap; ++sg) seg_start[sg] = i;
    }
}

cudaError_t launch_pair_segments(const uint32_t* tiles, const uint32_t* order, const uint32_t* n_dev,
                                 const uint32_t* pair_off, uint32_t* seg_start, int64_t seg_cap, int grid,
                                 cudaStream_t s) {
    pair_segments_kernel<<<grid, 256, 0, s>>>(tiles, order, n_dev, pair_off, seg_start,
                                              (uint32_t)std::min<int64_t>(seg_cap, 0xffffffffLL));
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ duplication
//
// Block b writes pairs [b DUP_SEG, (b + 1) DUP_SEG) (key = global tile id, value = cut position; a
// splat's tiles in row-major order), fully coalesced.  The entries covering the segment are
// seg_start[b] .. seg_start[b + 1] (the last one may continue into the next segment); they are
// staged in shared memory and every pair finds its entry by binary search over their offsets.

__global__ void __launch_bounds__(256) duplicate_kernel(const DevCam* __restrict__ cams, int n_cams,
                                                        const int64_t* __restrict__ cut_offsets, SplatBufs sb,
                                                        const uint32_t* __restrict__ order,
                                                        const uint32_t* __restrict__ n_order,
                                                        const uint32_t* __restrict__ pair_off,
                                                        const uint32_t* __restrict__ seg_start,
                                                        const uint32_t* __restrict__ n_pairs, int64_t cap_pairs,
                                                        uint32_t* __restrict__ n_pairs_kept,
                                                        uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                        uint32_t* __restrict__ hist, int hist_passes,
                                                        uint32_t* __restrict__ flags) {
    griddep_launch_dependents();
    griddep_wait();
    __shared__ uint32_t s_off[DUP_SEG + 1], s_m[DUP_SEG + 1], s_xy[DUP_SEG + 1], s_wtx[DUP_SEG + 1],
        s_tb[DUP_SEG + 1];
    __shared__ uint32_t s_hist[4][256];   // digit histograms of the tile keys for the tile sort
    const uint32_t P = *n_pairs;
    const uint32_t Pk = (int64_t)P > cap_pairs ? (uint32_t)cap_pairs : P;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *n_pairs_kept = Pk;
        if ((int64_t)P > cap_pairs) atomicOr(flags, FLAG_PAIRS_OVERFLOW);
    }
    const uint64_t p0 = (uint64_t)blockIdx.x * DUP_SEG;
    if (p0 >= Pk) return;
    const uint64_t p1 = min((uint64_t)Pk, p0 + DUP_SEG);
    const uint32_t V = *n_order;
    const uint32_t e0 = seg_start[blockIdx.x];
    const uint32_t e1 = p1 < Pk ? seg_start[blockIdx.x + 1] : V - 1;
    if (e0 >= V || e1 < e0) return;   // only after a failed scan (flagged)
    if (hist)
        for (int i = threadIdx.x; i < hist_passes * 256; i += blockDim.x) (&s_hist[0][0])[i] = 0;
    const int ne = (int)min(min(e1 - e0 + 1, (uint32_t)DUP_SEG + 1), V - e0);
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const uint32_t i = e0 + e;
        uint32_t m = __ldg(order + i);
        if (!H3DGS_IN(m, *sb.n_splats)) m = 0;   // checked build only
        const uint2 r = sb.rect[m];
        const int k = find_cam(cut_offsets, n_cams, m);
        s_off[e] = __ldg(pair_off + i);
        s_m[e] = m;
        s_xy[e] = (r.x & 0xffffu) | (r.y << 16);                                // x0 | y0 << 16
        s_wtx[e] = ((r.x >> 16) - (r.x & 0xffffu) + 1) | ((uint32_t)cams[k].tiles_x << 16);
        s_tb[e] = (uint32_t)cams[k].tile_base;
    }
    __syncthreads();
    for (uint64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        int lo = 0, hi = ne - 1;   // last entry whose first pair is <= p
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= p) lo = mid; else hi = mid - 1;
        }
        const uint32_t k = (uint32_t)(p - s_off[lo]);
        const uint32_t wtx = s_wtx[lo], xy = s_xy[lo];
        const uint32_t w = wtx & 0xffffu, ty = k / w, tx = k - ty * w;
        const uint32_t key = s_tb[lo] + ((xy >> 16) + ty) * (wtx >> 16) + (xy & 0xffffu) + tx;
        keys[p] = key;
        vals[p] = s_m[lo];
        if (hist)
            for (int q = 0; q < hist_passes; ++q) atomicAdd(&s_hist[q][(key >> (8 * q)) & 255u], 1u);
    }
    if (hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < hist_passes * 256; i += blockDim.x) {
            const uint32_t c = (&s_hist[0][0])[i];
            if (c) atomicAdd(hist + i, c);
        }
    }
}

cudaError_t launch_duplicate(const DevCam* cams, int n_cams, const int64_t* cut_offsets, const SplatBufs& sb,
                             const uint32_t* order, const uint32_t* n_order, const uint32_t* pair_off,
                             const uint32_t* seg_start, const uint32_t* n_pairs, int64_t cap_pairs,
                             uint32_t* n_pairs_kept, uint32_t* keys, uint32_t* vals, uint32_t* hist, int hist_passes,
                             uint32_t* flags, cudaStream_t s) {
    const int64_t blocks = std::max<int64_t>(1, (cap_pairs + DUP_SEG - 1) / DUP_SEG);
    if (hist_passes < 0 || hist_passes > 4) return cudaErrorInvalidValue;
    return launch_dependent(duplicate_kernel, dim3((unsigned)blocks), dim3(256), s, cams, n_cams, cut_offsets, sb, order,
                            n_order, pair_off, seg_start, n_pairs, cap_pairs, n_pairs_kept, keys, vals, hist,
                            hist_passes, flags);
}

H3DGS_CHECK_READER(check_read_sort)

}  // namespace h3dgs
