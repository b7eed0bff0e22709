// Single-pass exclusive scan across thread blocks with decoupled look-back (Merrill and Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016).
//
// Blocks take their index from a ticket counter, so a block only ever waits for blocks that took
// a ticket earlier and are therefore running.  Each block publishes its aggregate, then warp 0 reads
// the status words of up to 32 earlier blocks at a time, newest first, until it meets an inclusive
// prefix.  Every wait on a word that is not yet published is bounded; a wait that gives up sets
// FLAG_WAIT_TIMEOUT in the device flag word and the result is invalid (the context stays usable).
//
// Grouped variant (gsum != NULL), for launches whose blocks are all resident at once: every block
// also adds its aggregate to its group's sum (LB_GROUP blocks per group) and raises the group's
// completion counter; a block's prefix is then the sums of the complete earlier groups plus the
// aggregates of the earlier blocks of its group, independent loads instead of a chain of inclusive
// prefixes that grows with the block's position.
#pragma once

#include "internal.cuh"

namespace h3dgs {

constexpr unsigned long long LB_AGG = 1ull << 62;   // status word: the block's own aggregate
constexpr unsigned long long LB_INC = 1ull << 63;   // status word: inclusive prefix up to the block
constexpr unsigned long long LB_VAL = (1ull << 62) - 1;
constexpr int LB_SPIN_LIMIT = 1 << 20;
constexpr int LB_GROUP = 32;   // blocks per group of the grouped variant (one warp reads a group)

struct Lookback {
    unsigned long long* status;   // one word per block, zero before the launch
    uint32_t* ticket;             // zero before the launch
    uint32_t* flags;              // device flag word
    unsigned long long* gsum = nullptr;   // grouped variant: [groups] sums, zero before the launch
    uint32_t* gcnt = nullptr;             // grouped variant: [groups] completion counters, zero before
};

// Workspace words of a look-back over `blocks` blocks after the LB_HEADER_WORDS header: the status
// words, then the group sums and counters of the grouped variant.
__host__ __device__ inline size_t lb_body_words(int64_t blocks) {
    const int64_t groups = (blocks + LB_GROUP - 1) / LB_GROUP;
    return 2 * (size_t)blocks + 3 * (size_t)groups;
}
// A Lookback over the workspace `work` (LB_HEADER_WORDS + lb_body_words(blocks) words); grouped
// when every block of the launch is resident at once.
inline Lookback lb_make(uint32_t* work, int64_t blocks, bool grouped, uint32_t* flags) {
    Lookback lb;
    lb.status = reinterpret_cast<unsigned long long*>(work + LB_HEADER_WORDS);
    lb.ticket = work;
    lb.flags = flags;
    if (grouped) {
        lb.gsum = reinterpret_cast<unsigned long long*>(work + LB_HEADER_WORDS + 2 * blocks);
        lb.gcnt = work + LB_HEADER_WORDS + 2 * blocks + 2 * ((blocks + LB_GROUP - 1) / LB_GROUP);
    }
    return lb;
}

__device__ __forceinline__ unsigned long long lb_load(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void lb_store(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// The block's index in ticket order (all threads).
__device__ __forceinline__ uint32_t lb_ticket(const Lookback& lb, uint32_t* s_slot) {
    if (threadIdx.x == 0) *s_slot = atomicAdd(lb.ticket, 1u);
    __syncthreads();
    return *s_slot;
}

// Exclusive prefix of block b from its aggregate agg (all threads call it; the result is the same in
// every thread).  s_slot: one shared 64-bit word.
// Publishes block b's aggregate without waiting for its prefix (thread 0; for a block that writes
// nothing).  Later blocks sum it on their way back as they sum any published aggregate.
__device__ __forceinline__ void lb_publish(const Lookback& lb, uint32_t b, unsigned long long agg) {
    if (threadIdx.x != 0) return;
    lb_store(lb.status + b, (b == 0 ? LB_INC : LB_AGG) | agg);
    if (lb.gsum) {
        const uint32_t g = b / LB_GROUP;
        atomicAdd(lb.gsum + g, agg);
        __threadfence();
        atomicAdd(lb.gcnt + g, 1u);
    }
}

__device__ __forceinline__ unsigned long long lb_prefix(const Lookback& lb, uint32_t b, unsigned long long agg,
                                                        unsigned long long* s_slot) {
    if (threadIdx.x == 0) lb_store(lb.status + b, (b == 0 ? LB_INC : LB_AGG) | agg);
    if (lb.gsum) {
        const uint32_t g = b / LB_GROUP;
        if (threadIdx.x == 0) {
            atomicAdd(lb.gsum + g, agg);
            __threadfence();
            atomicAdd(lb.gcnt + g, 1u);
        }
        if (b > 0 && threadIdx.x < 32) {
            const int lane = threadIdx.x;
            unsigned long long x = 0;
            for (uint32_t q = lane; q < g; q += 32) {   // complete earlier groups
                uint32_t c;
                int spins = 0;
                while (true) {
                    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(lb.gcnt + q) : "memory");
                    if (c >= (uint32_t)LB_GROUP || spins >= LB_SPIN_LIMIT) break;
                    if (++spins > 32) __nanosleep(64);
                }
                if (c < (uint32_t)LB_GROUP) atomicOr(lb.flags, FLAG_WAIT_TIMEOUT);
                x += lb_load(lb.gsum + q);
            }
            const uint32_t k = g * LB_GROUP + lane;   // earlier blocks of this group
            if (k < b) {
                unsigned long long v = lb_load(lb.status + k);
                int spins = 0;
                while ((v >> 62) == 0 && spins < LB_SPIN_LIMIT) {
                    if (++spins > 32) __nanosleep(64);
                    v = lb_load(lb.status + k);
                }
                if ((v >> 62) == 0) atomicOr(lb.flags, FLAG_WAIT_TIMEOUT);
                else x += v & LB_VAL;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0) *s_slot = x;
        }
    } else if (b > 0 && threadIdx.x < 32) {
        const int lane = threadIdx.x;
        unsigned long long prefix = 0;
        int64_t j = (int64_t)b - 1;
        bool done = false;
        while (!done) {
            const int64_t k = j - lane;
            unsigned long long v = LB_INC;   // before block 0: an inclusive zero
            if (k >= 0) {
                v = lb_load(lb.status + k);
                int spins = 0;
                while ((v >> 62) == 0 && spins < LB_SPIN_LIMIT) {
                    if (++spins > 32) __nanosleep(64);
                    v = lb_load(lb.status + k);
                }
                if ((v >> 62) == 0) {
                    atomicOr(lb.flags, FLAG_WAIT_TIMEOUT);
                    v = LB_INC;
                }
            }
            const uint32_t inc = __ballot_sync(0xffffffffu, (v & LB_INC) != 0);
            const int first = inc ? __ffs(inc) - 1 : 31;
            unsigned long long x = lane <= first ? (v & LB_VAL) : 0ull;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            prefix += x;
            done = inc != 0;
            j -= 32;
        }
        if (lane == 0) {
            lb_store(lb.status + b, LB_INC | ((prefix + agg) & LB_VAL));
            *s_slot = prefix;
        }
    }
    __syncthreads();
    const unsigned long long p = b == 0 ? 0ull : *s_slot;
    __syncthreads();
    return p;
}

// Exclusive scan over the threads of a block of NT threads (NT/32 <= 32); *total gets the block sum.
template <int NT>
__device__ __forceinline__ unsigned long long lb_block_scan(unsigned long long x, unsigned long long* s_warp,
                                                            unsigned long long* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    unsigned long long before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        const unsigned long long s = s_warp[w];
        before += w < warp ? s : 0ull;
        all += s;
    }
    __syncthreads();
    *total = all;
    return before + inc - x;
}

}  // namespace h3dgs
