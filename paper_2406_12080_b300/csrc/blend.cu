// Per-tile front-to-back blending (a7), with long tile lists split into chunks.
//
// Per pixel and splat, in list order (tile list = (depth, cut position) order):
//   G = 2^(ca dx^2 + cb dx dy + cc dy^2)                (conic pre-scaled by -log2(e)/2)
//   alpha_n = min(c, o_n G),  alpha_p = min(c, o_p G)
//   alpha'  = 1 - (1 - alpha_p)^(1/K)                   (Eq. alphap; K = 2: alpha_p / (1 + sqrt(1 - alpha_p)))
//   alpha   = (1 - t) alpha_n + t alpha'                (t = parent weight; t = 0 skips alpha')
//   skip alpha < alpha_floor; stop before T (1 - alpha) < t_min; C += colour alpha T.
// The per-pixel decision quantities (dx, dy, exponent, alpha, T) use a fixed fp32 order.
//
// Street scenes put thousands of splats behind some pixels (near the vanishing point), so a
// one-CTA-per-tile blend is bounded by its longest list.  A list of L > `chunk` entries is cut into
// ceil(L / chunk) chunks of near-equal length that run as separate CTAs ("items"):
//   producers (chunks 0 .. nch - 2 of split tiles) walk their chunk from T = 1 with the exact
//             skip/stop rules and hand on the chunk's product of (1 - alpha) over its contributors
//             (0 if the walk stopped), so that every chunk's incoming transmittance T_in is a product
//             of the earlier chunks' products; the local colour, end transmittance and last
//             contributor go to a per-(item, pixel) scratch;
//   consumers (chunks 1 .. nch - 1) and single-chunk tiles walk their entries from T_in with the
//             exact rules.  A pixel of a middle chunk whose T_in times the chunk's product is above
//             t_min by more than the rounding of the product cannot stop inside the chunk; there the
//             walk from T_in takes the same decisions as the producer's walk from 1, and its colour,
//             end transmittance and depth are the local ones times T_in, so the consumer takes those
//             instead of walking.  Single-chunk tiles write the pixel directly, chunks of split tiles
//             write (colour, T at the end, last contributor) to the scratch kept for the adjoint;
//   combine   by the consumer of each split tile's last chunk, after a bounded wait on the tile's other
//             consumers (all taken before it): per pixel, colour = sum of the chunks, T_final and the
//             last contributor from the chunk where the walk stopped.
// A chunk whose T_in is already below t_min adds nothing (the walk stopped in an earlier chunk).
//
// Optional outputs (appendix, depth regularisation and exposure optimisation): the expected depth
// sum(T alpha z), accumulated like a fourth colour channel with the splat's view depth z and no
// background term, and the camera's 3x4 exposure affine applied to the pixel colour,
// out = E [C + T bg | 1].
#include <algorithm>

#include "internal.cuh"
#include "lookback.cuh"

namespace h3dgs {

// alpha of one (pixel, splat) pair, fixed fp32 order; K (child count) is read only when t != 0
__device__ __forceinline__ float pair_alpha(float px, float py, const float4 a, const float4 b, const float4* c,
                                            float clampv) {
    const float dx = fsub(px, a.x), dy = fsub(py, a.y);
    const float h = ffma(a.z, dx, fmul(a.w, dy));
    const float g = fmul(fmul(b.x, dy), dy);
    const float p2 = ffma(dx, h, g);
    const float G = ex2_approx(p2);
    const float an = fminf(clampv, fmul(b.y, G));
    if (b.w == 0.0f) return an;
    const float ap = fminf(clampv, fmul(b.z, G));
    return ffma(b.w, alpha_prime(ap, c->w), fmul(fsub(1.0f, b.w), an));
}

// alpha of two pixels of the same column (rows py.x, py.y) for one splat, in the same fixed fp32 order
// as pair_alpha per pixel (the paired instructions round every element like the scalar ones)
__device__ __forceinline__ float2 pair_alpha2(float px, float2 py, const float4 a, const float4 b, const float4* c,
                                              float clampv) {
    const float dx = fsub(px, a.x);
    const float2 dy = __fadd2_rn(py, make_float2(-a.y, -a.y));
    const float2 h = __ffma2_rn(make_float2(a.z, a.z), make_float2(dx, dx), __fmul2_rn(make_float2(a.w, a.w), dy));
    const float2 g = __fmul2_rn(__fmul2_rn(make_float2(b.x, b.x), dy), dy);
    const float2 p2 = __ffma2_rn(make_float2(dx, dx), h, g);
    const float2 G = make_float2(ex2_approx(p2.x), ex2_approx(p2.y));
    const float2 xn = __fmul2_rn(make_float2(b.y, b.y), G);
    const float2 an = make_float2(fminf(clampv, xn.x), fminf(clampv, xn.y));
    if (b.w == 0.0f) return an;
    const float2 xp = __fmul2_rn(make_float2(b.z, b.z), G);
    const float K = c->w;
    const float2 apr = make_float2(alpha_prime(fminf(clampv, xp.x), K), alpha_prime(fminf(clampv, xp.y), K));
    const float omw = fsub(1.0f, b.w);
    return __ffma2_rn(make_float2(b.w, b.w), apr, __fmul2_rn(make_float2(omw, omw), an));
}

// This thread's two pixels of the tile and the tile's camera.
template <int TW, int TH>
struct TileGeom2 {
    int ox, oy;                 // tile's pixel origin
    int px_i, py_i0, py_i1;     // the two pixels (same column)
    int slot0, slot1;           // their indices in the tile (row-major), for the per-pixel scratch
    bool in0, in1;
    float px;
    float2 py;
    const DevCam* cam;
};

template <int TW, int TH>
__device__ __forceinline__ TileGeom2<TW, TH> tile_geom2(const DevCam* __restrict__ cams, int n_cams, int64_t tile) {
    int lo = 0, hi = n_cams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cams[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    TileGeom2<TW, TH> g;
    g.cam = cams + lo;
    const int local = (int)(tile - g.cam->tile_base);
    g.ox = (local % g.cam->tiles_x) * TW;
    g.oy = (local / g.cam->tiles_x) * TH;
    int lx, ly0;
    tile_pixel2<TW, TH>(threadIdx.x, lx, ly0);
    g.px_i = g.ox + lx;
    g.py_i0 = g.oy + ly0;
    g.py_i1 = g.py_i0 + 4;
    g.slot0 = ly0 * TW + lx;
    g.slot1 = (ly0 + 4) * TW + lx;
    g.in0 = g.px_i < g.cam->width && g.py_i0 < g.cam->height;
    g.in1 = g.px_i < g.cam->width && g.py_i1 < g.cam->height;
    g.px = (float)g.px_i + 0.5f;
    g.py = make_float2((float)g.py_i0 + 0.5f, (float)g.py_i1 + 0.5f);
    return g;
}

// ------------------------------------------------------------------------------------ plan

// The plan: the tile ranges decoded, chunk counts per tile, their exclusive scan (single pass, decoupled look-back), the full
// (tile, chunk) item list (used by the blend and the adjoint) and the work queue of the blend:
//   producers  chunks 0 .. nch - 2 of split tiles, blended from T = 1; each hands on its (1 - alpha)
//              product;
//   singles    tiles of one chunk;
//   consumers  chunks 1 .. nch - 1 of split tiles, blended from the product of the earlier chunks.
// Per tile the scan carries X = nch - 1 (split tiles) and Y = [nch == 1] packed in one word; the item
// offset is t + prefix(X), the producer and consumer offsets prefix(X), the single offset prefix(Y).
constexpr int PL_THREADS = 256;
constexpr int PL_IPT = 1;   // one tile per thread: 32 blocks at 1080p (4 tiles per thread left 8 blocks)
constexpr int PL_TILE = PL_THREADS * PL_IPT;

__global__ void __launch_bounds__(PL_THREADS) blend_plan_kernel(int2* __restrict__ ranges, int64_t n_tiles,
                                                                int chunk, const uint32_t* __restrict__ n_pairs,
                                                                int32_t* __restrict__ tile_item0,
                                                                int32_t* __restrict__ tile_nch,
                                                                int2* __restrict__ items, int64_t item_cap,
                                                                uint32_t* __restrict__ q_prod,
                                                                uint32_t* __restrict__ q_single,
                                                                uint32_t* __restrict__ q_cons,
                                                                uint32_t* __restrict__ counts /* items, X, Y, Z */,
                                                                Lookback lb) {
    griddep_launch_dependents();
    griddep_wait();
    __shared__ uint32_t s_ticket;
    __shared__ unsigned long long s_slot, s_warp[PL_THREADS / 32];
    // the automatic chunk: with the split threshold of the frame, longer lists go in chunks of
    // BLEND_AUTO_CHUNK
    int split_min = chunk;
    if (chunk <= 0) {
        chunk = BLEND_AUTO_CHUNK;
        split_min = blend_auto_split(*n_pairs, n_tiles);
    }
    const uint32_t b = lb_ticket(lb, &s_ticket);
    const int64_t base = (int64_t)b * PL_TILE;
    if (base >= n_tiles) return;
    int nch[PL_IPT];
    unsigned long long sum = 0;
#pragma unroll
    for (int q = 0; q < PL_IPT; ++q) {
        const int64_t t = base + (int64_t)threadIdx.x * PL_IPT + q;
        nch[q] = 0;
        if (t < n_tiles) {
            // the tile sort leaves {~first, last + 1} ({0, 0} for a tile without pairs): decoded here,
            // in place, for the blend and the adjoint
            int2 r = ranges[t];
            r = r.y == 0 ? make_int2(0, 0) : make_int2(~r.x, r.y);
            ranges[t] = r;
            const int len = r.y - r.x;
            nch[q] = len <= split_min ? 1 : (len + chunk - 1) / chunk;
            sum += ((unsigned long long)(nch[q] - 1) << 31) | (unsigned long long)(nch[q] == 1);
        }
    }
    unsigned long long agg;
    const unsigned long long before = lb_block_scan<PL_THREADS>(sum, s_warp, &agg);
    const unsigned long long pre = lb_prefix(lb, b, agg, &s_slot) + before;
    int64_t offX = (int64_t)(pre >> 31), offY = (int64_t)(pre & 0x7fffffffull);
#pragma unroll
    for (int q = 0; q < PL_IPT; ++q) {
        const int64_t t = base + (int64_t)threadIdx.x * PL_IPT + q;
        if (t < n_tiles) {
            const int n = nch[q];
            const int64_t offF = t + offX;
            tile_item0[t] = (int32_t)offF;
            tile_nch[t] = n;
            for (int c = 0; c < n; ++c) {
                const int64_t it = offF + c;
                if (it >= item_cap) break;
                items[it] = make_int2((int)t, c);
                if (n == 1) q_single[offY] = (uint32_t)it;
                else {
                    if (c < n - 1) q_prod[offX + c] = (uint32_t)it;
                    if (c >= 1) q_cons[offX + c - 1] = (uint32_t)it;
                }
            }
            if (t + 1 == n_tiles) {
                const int64_t X = offX + n - 1, Y = offY + (n == 1);
                const int64_t F = n_tiles + X;
                const bool fits = F <= item_cap;
                counts[0] = (uint32_t)min(F, item_cap);
                counts[1] = fits ? (uint32_t)X : 0u;   // an overflowing plan blends nothing (flagged)
                counts[2] = fits ? (uint32_t)Y : 0u;
                counts[3] = fits ? (uint32_t)(n_tiles - Y) : 0u;
            }
            offX += n - 1;
            offY += (n == 1);
        }
    }
}

// ------------------------------------------------------------------------------------ passes

// Scratch per (item, pixel), struct-of-arrays over pixels: Tc, C0, C1, C2, Tend, last.
struct Scratch {
    float* Tc;     // product of (1 - alpha) over the chunk's contributors (0 once the walk stopped)
    float* C;      // [3] colour of the chunk
    float* Tend;   // T after the chunk's walk (stop applied)
    int32_t* last; // list position (within the tile) after the chunk's last contributor, or -1
    float* D;      // expected depth of the chunk (depth output only)
};

// One pixel's colour C + T bg, through the camera's exposure affine E (row-major 3x4) when given.
__device__ __forceinline__ void write_pixel(float* img, int64_t plane, float T, float C0, float C1, float C2,
                                            const DevOpts& o, const float* __restrict__ E) {
    const float r = fmaf(T, o.bg[0], C0), g = fmaf(T, o.bg[1], C1), b = fmaf(T, o.bg[2], C2);
    if (E) {
        img[0] = fmaf(E[0], r, fmaf(E[1], g, fmaf(E[2], b, E[3])));
        img[plane] = fmaf(E[4], r, fmaf(E[5], g, fmaf(E[6], b, E[7])));
        img[2 * plane] = fmaf(E[8], r, fmaf(E[9], g, fmaf(E[10], b, E[11])));
    } else {
        img[0] = r;
        img[plane] = g;
        img[2 * plane] = b;
    }
}

// Walk of one item over list entries [begin, end) for this thread's two pixels with the exact
// skip/stop rules.  DEPTH: the expected depth Dp is accumulated as a fourth channel.  SAVE: track the
// last contributor (kept for the adjoint).
//
// The per-entry work is arranged to keep the per-pixel decisions off the critical ALU pipe while
// producing bit-identical results to the direct formulation:
//   * each pixel has a floor threshold fl (alpha_floor, or +inf once the pixel has stopped or lies
//     outside the image), so one compare per pixel both applies the 1/255 skip and drops finished
//     pixels;
//   * a pixel that does not take the entry gets alpha_eff = 0, and T (1 - alpha_eff) = T and
//     C + c alpha_eff T = C hold exactly, so T and the colours are updated with paired fp32
//     arithmetic and no selects;
//   * the transmittance stop can only happen at a pixel that takes the entry, at most once per
//     pixel, so it is handled in a warp-uniform branch that is rarely entered: it freezes the
//     pixel (fl = +inf) and undoes the entry for it (stop before the splat).
template <int TW, int TH, bool COUNT, bool DEPTH, bool SAVE>
__device__ __forceinline__ void blend_walk2(const TileGeom2<TW, TH>& g, const uint32_t* __restrict__ list,
                                            const float4* __restrict__ splat, const uint32_t* __restrict__ n_spl,
                                            int begin, int end, int list0,
                                            float clampv, float afloor, float tmin, float4* s_a, float4* s_b,
                                            float4* s_c, uint32_t* s_m, float* s_d, float4* s_box, float2& T, float2& C0,
                                            float2& C1, float2& C2, float2& Dp, int2& last, bool& done0, bool& done1,
                                            unsigned int& evals, unsigned int& evals_i, unsigned int& contribs,
                                            unsigned int& contribs_i) {
    constexpr int NT2 = TW * TH / 2, NW = NT2 / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float INF = __int_as_float(0x7f800000);
    float2 fl = make_float2(done0 ? INF : afloor, done1 ? INF : afloor);
    for (int b0 = begin; b0 < end; b0 += NT2) {
        // the warp's live pixels' bounding box (pixel centres): entries that cannot reach alpha_floor
        // inside it are skipped by the warp mask (its stopped pixels no longer matter)
        {
            const bool any_live = !(done0 && done1);
            const int ix = g.px_i;
            const int iy_lo = !done0 ? g.py_i0 : g.py_i1, iy_hi = !done1 ? g.py_i1 : g.py_i0;
            const int xmin = __reduce_min_sync(0xffffffffu, any_live ? ix : 0x7fffffff);
            const int xmax = __reduce_max_sync(0xffffffffu, any_live ? ix : -1);
            const int ymin = __reduce_min_sync(0xffffffffu, any_live ? iy_lo : 0x7fffffff);
            const int ymax = __reduce_max_sync(0xffffffffu, any_live ? iy_hi : -1);
            if (lane == 0)
                s_box[warp] = xmax < 0 ? make_float4(1.0f, 1.0f, -1.0f, -1.0f)
                                       : make_float4((float)xmin + 0.5f, (float)ymin + 0.5f, (float)xmax + 0.5f,
                                                     (float)ymax + 0.5f);
        }
        if (__syncthreads_count(done0 && done1) == NT2) break;
        const int n = min(NT2, end - b0);
        if ((int)threadIdx.x < n) {
            uint32_t s = __ldg(list + b0 + threadIdx.x);
            if (!H3DGS_IN(s, *n_spl)) s = 0;   // checked build only
            const float4 a = __ldg(splat + SPLAT_F4 * (int64_t)s);
            const float4 bb = __ldg(splat + SPLAT_F4 * (int64_t)s + 1);
            const float4 d = __ldg(splat + SPLAT_F4 * (int64_t)s + 3);
            s_a[threadIdx.x] = a;
            s_b[threadIdx.x] = bb;
            s_c[threadIdx.x] = __ldg(splat + SPLAT_F4 * (int64_t)s + 2);
            uint32_t wm = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const float4 bx = s_box[w];
                if (bx.x <= bx.z && rect_reach(a, bb.x, d, bx.x, bx.y, bx.z, bx.w)) wm |= 1u << w;
            }
            s_m[threadIdx.x] = wm;
            if (DEPTH) s_d[threadIdx.x] = d.w;
        }
        __syncthreads();
        if (__any_sync(0xffffffffu, !(done0 && done1))) {
            for (int base = 0; base < n; base += 32) {
                const uint32_t mm = (base + lane < n) ? s_m[base + lane] : 0u;
                uint32_t bits = __ballot_sync(0xffffffffu, (mm >> warp) & 1u);
                while (bits) {
                    const int j = base + __ffs(bits) - 1;
                    bits &= bits - 1;
                    if (COUNT) {
                        evals += (unsigned)!done0 + (unsigned)!done1;
                        if (s_b[j].w != 0.0f) evals_i += (unsigned)!done0 + (unsigned)!done1;
                    }
                    const float2 alpha = pair_alpha2(g.px, g.py, s_a[j], s_b[j], &s_c[j], clampv);
                    bool take0 = alpha.x >= fl.x, take1 = alpha.y >= fl.y;
                    float2 ae = make_float2(take0 ? alpha.x : 0.0f, take1 ? alpha.y : 0.0f);
                    float2 Tn = __fmul2_rn(T, __fadd2_rn(make_float2(1.0f, 1.0f), make_float2(-ae.x, -ae.y)));
                    const bool stop0 = take0 && Tn.x < tmin, stop1 = take1 && Tn.y < tmin;
                    if (__any_sync(0xffffffffu, stop0 || stop1)) {
                        // at most once per pixel: the pixel finishes here
                        if (stop0) {
                            done0 = true;
                            fl.x = INF;
                            ae.x = 0.0f; Tn.x = T.x; take0 = false;
                        }
                        if (stop1) {
                            done1 = true;
                            fl.y = INF;
                            ae.y = 0.0f; Tn.y = T.y; take1 = false;
                        }
                    }
                    {
                        const float2 w = __fmul2_rn(ae, T);
                        const float4 c = s_c[j];
                        C0 = __ffma2_rn(make_float2(c.x, c.x), w, C0);
                        C1 = __ffma2_rn(make_float2(c.y, c.y), w, C1);
                        C2 = __ffma2_rn(make_float2(c.z, c.z), w, C2);
                        if (DEPTH) Dp = __ffma2_rn(make_float2(s_d[j], s_d[j]), w, Dp);
                        if (SAVE) {
                            const int pos = b0 + j + 1 - list0;
                            last = make_int2(take0 ? pos : last.x, take1 ? pos : last.y);
                        }
                        if (COUNT) {
                            contribs += (unsigned)take0 + (unsigned)take1;
                            if (s_b[j].w != 0.0f) contribs_i += (unsigned)take0 + (unsigned)take1;
                        }
                    }
                    T = Tn;
                }
                if (__all_sync(0xffffffffu, done0 && done1)) break;
            }
        }
    }
}

// The blend: one CTA per queue entry, in ticket order (a CTA holding ticket k is running, and every
// entry before k has been taken by a running CTA).  Producers never wait; a consumer waits until the
// producers of its tile have published their products (per-tile counter, bounded wait), which were
// all taken before it.  TW x TH / 2 threads, two pixels each.  COUNT: count the (pixel, splat)
// evaluations into n_evals (profiling only; the count costs instructions in the innermost loop).
// DEPTH: also the expected depth (depth != NULL).  SAVE: also the per-pixel state the adjoint reads
// (final transmittance, contributor count; T_final and n_contrib != NULL).
template <int TW, int TH, bool COUNT, bool DEPTH, bool SAVE>
__global__ void __launch_bounds__(TW * TH / 2, 12) blend_queue_kernel(const DevCam* __restrict__ cams, int n_cams, DevOpts o,
                                                                  const int2* __restrict__ ranges,
                                                                  const uint32_t* __restrict__ list,
                                                                  const float4* __restrict__ splat,
                                                                  const uint32_t* __restrict__ n_spl,
                                                                  const int2* __restrict__ items,
                                                                  const uint32_t* __restrict__ q_prod,
                                                                  const uint32_t* __restrict__ q_single,
                                                                  const uint32_t* __restrict__ q_cons,
                                                                  const uint32_t* __restrict__ counts,
                                                                  const int32_t* __restrict__ tile_item0,
                                                                  const int32_t* __restrict__ tile_nch, Scratch sc,
                                                                  uint32_t* __restrict__ ticket,
                                                                  uint32_t* __restrict__ tile_done,
                                                                  uint32_t* __restrict__ cons_done,
                                                                  float* __restrict__ images,
                                                                  float* __restrict__ depth,
                                                                  const float* __restrict__ exposure,
                                                                  float* __restrict__ T_final,
                                                                  int32_t* __restrict__ n_contrib,
                                                                  unsigned long long* __restrict__ n_evals,
                                                                  uint32_t* __restrict__ flags) {
    griddep_launch_dependents();
    griddep_wait();
    constexpr int NT = TW * TH, NT2 = NT / 2;
    __shared__ float4 s_a[NT2], s_b[NT2], s_c[NT2];
    __shared__ uint32_t s_m[NT2];
    __shared__ float s_d[DEPTH ? NT2 : 1];
    __shared__ float4 s_box[NT2 / 32];
    __shared__ unsigned int s_evals[5];
    __shared__ uint32_t s_k;
    if (threadIdx.x == 0) s_k = atomicAdd(ticket, 1u);
    if (threadIdx.x < 5) s_evals[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t k = s_k;
    const uint32_t X = counts[1], Y = counts[2];
    int role;   // 0: producer, 1: single, 2: consumer
    uint32_t item;
    if (k < X) { role = 0; item = q_prod[k]; }
    else if (k < X + Y) { role = 1; item = q_single[k - X]; }
    else if (k < 2 * X + Y) { role = 2; item = q_cons[k - X - Y]; }
    else return;
    if (!H3DGS_IN(item, counts[0])) return;   // checked build only
    const int2 it = items[item];
    const int64_t tile = it.x;
    const int nch = tile_nch[tile];
    const TileGeom2<TW, TH> g = tile_geom2<TW, TH>(cams, n_cams, tile);
    const int2 r = ranges[tile];
    const int begin = chunk_begin(r, nch, it.y);
    const int end = chunk_begin(r, nch, it.y + 1);
    const int64_t s0 = (int64_t)item * NT + g.slot0, s1 = (int64_t)item * NT + g.slot1;
    const int lane = threadIdx.x & 31;
    float2 T = make_float2(1.0f, 1.0f);
    float2 Tc = T;                      // the producer's product of this chunk (middle chunks)
    bool short0 = false, short1 = false;
    if (role == 2) {
        // wait for the tile's nch - 1 producers, then T_in = product of the earlier chunks' products
        if (threadIdx.x == 0) wait_geq(tile_done + tile, (uint32_t)(nch - 1), QUEUE_SPIN_LIMIT, flags);
        __syncthreads();
        const int64_t i0 = tile_item0[tile];
        for (int c = 0; c < it.y; ++c)
            T = __fmul2_rn(T, make_float2(__ldcg(sc.Tc + (i0 + c) * NT + g.slot0), __ldcg(sc.Tc + (i0 + c) * NT + g.slot1)));
        if (it.y + 1 < nch) {
            // T_in Tc >= t_min (1 + 4 len u) (u = 2^-24): the sequential products from T_in differ from
            // T_in Tc by at most 2 len roundings, so no T (1 - alpha) of the chunk falls below t_min (a
            // product the local walk stopped on is 0 and never passes)
            Tc = make_float2(__ldcg(sc.Tc + s0), __ldcg(sc.Tc + s1));
            const float thr = fmul(o.t_min, ffma((float)(end - begin), 2.384185791015625e-7f, 1.0f));
            const float2 P = __fmul2_rn(T, Tc);
            short0 = g.in0 && P.x >= thr;
            short1 = g.in1 && P.y >= thr;
        }
    }
    float2 C0 = make_float2(0.0f, 0.0f), C1 = C0, C2 = C0, Dp = C0;
    int2 last = make_int2(-1, -1);
    unsigned int evals = 0, evals_i = 0, contribs = 0, contribs_i = 0;
    // while counting, every pixel walks (the counts are those of the sequential walk) and the shortcut's
    // values replace the walk's afterwards, so that the image does not depend on the counting
    const float2 Tin = T;
    bool done0 = !g.in0 || T.x < o.t_min || (!COUNT && short0), done1 = !g.in1 || T.y < o.t_min || (!COUNT && short1);
    blend_walk2<TW, TH, COUNT, DEPTH, SAVE>(g, list, splat, n_spl, begin, end, r.x, o.alpha_clamp, o.alpha_floor,
                                            o.t_min, s_a, s_b, s_c, s_m, s_d, s_box, T, C0, C1, C2, Dp, last, done0,
                                            done1, evals, evals_i, contribs, contribs_i);
    if (COUNT) {
        for (int off = 16; off > 0; off >>= 1) {
            evals += __shfl_down_sync(0xffffffffu, evals, off);
            evals_i += __shfl_down_sync(0xffffffffu, evals_i, off);
            contribs += __shfl_down_sync(0xffffffffu, contribs, off);
            contribs_i += __shfl_down_sync(0xffffffffu, contribs_i, off);
        }
        // the middle producers' walks are repeated by their consumers while counting: counted apart,
        // as extra work
        const bool counted = role != 0 || it.y == 0;
        if (lane == 0) {
            atomicAdd(&s_evals[counted ? 0 : 1], evals);
            if (counted) {
                atomicAdd(&s_evals[2], evals_i);
                atomicAdd(&s_evals[3], contribs);
                atomicAdd(&s_evals[4], contribs_i);
            }
        }
    }
    if (role == 0) {
        // the local walk (the first chunk's is final) and the product handed to the later chunks:
        // 0 once the walk stopped
        sc.C[3 * s0 + 0] = C0.x; sc.C[3 * s0 + 1] = C1.x; sc.C[3 * s0 + 2] = C2.x;
        sc.C[3 * s1 + 0] = C0.y; sc.C[3 * s1 + 1] = C1.y; sc.C[3 * s1 + 2] = C2.y;
        sc.Tend[s0] = T.x;
        sc.Tend[s1] = T.y;
        if (SAVE) {
            sc.last[s0] = last.x;
            sc.last[s1] = last.y;
        }
        if (DEPTH) {
            sc.D[s0] = Dp.x;
            sc.D[s1] = Dp.y;
        }
        sc.Tc[s0] = (done0 && g.in0) ? 0.0f : T.x;
        sc.Tc[s1] = (done1 && g.in1) ? 0.0f : T.y;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(tile_done + tile, 1u);
    } else {
        __syncthreads();
    }
    if (COUNT && threadIdx.x < 5 && s_evals[threadIdx.x])
        atomicAdd(n_evals + threadIdx.x, (unsigned long long)s_evals[threadIdx.x]);
    if (role == 0) return;
    if (nch > 1) {
        // pixels that take the producer's walk: its local values times T_in (without counting, T still
        // holds T_in there)
        const float2 T0 = COUNT ? Tin : T;
        // checked build, while counting: the walk from T_in did not stop and ended on the producer's
        // last contributor
        if (COUNT && short0) H3DGS_HOLDS(!done0 && (!SAVE || last.x == __ldcg(sc.last + s0)));
        if (COUNT && short1) H3DGS_HOLDS(!done1 && (!SAVE || last.y == __ldcg(sc.last + s1)));
        if (short0) {
            C0.x = fmul(T0.x, __ldcg(sc.C + 3 * s0 + 0));
            C1.x = fmul(T0.x, __ldcg(sc.C + 3 * s0 + 1));
            C2.x = fmul(T0.x, __ldcg(sc.C + 3 * s0 + 2));
            if (SAVE) last.x = __ldcg(sc.last + s0);
            if (DEPTH) Dp.x = fmul(T0.x, __ldcg(sc.D + s0));
            T.x = fmul(T0.x, Tc.x);
        }
        if (short1) {
            C0.y = fmul(T0.y, __ldcg(sc.C + 3 * s1 + 0));
            C1.y = fmul(T0.y, __ldcg(sc.C + 3 * s1 + 1));
            C2.y = fmul(T0.y, __ldcg(sc.C + 3 * s1 + 2));
            if (SAVE) last.y = __ldcg(sc.last + s1);
            if (DEPTH) Dp.y = fmul(T0.y, __ldcg(sc.D + s1));
            T.y = fmul(T0.y, Tc.y);
        }
        sc.C[3 * s0 + 0] = C0.x; sc.C[3 * s0 + 1] = C1.x; sc.C[3 * s0 + 2] = C2.x;
        sc.C[3 * s1 + 0] = C0.y; sc.C[3 * s1 + 1] = C1.y; sc.C[3 * s1 + 2] = C2.y;
        sc.Tend[s0] = T.x;
        sc.Tend[s1] = T.y;
        if (SAVE) {
            sc.last[s0] = last.x;
            sc.last[s1] = last.y;
        }
        if (DEPTH) {
            sc.D[s0] = Dp.x;
            sc.D[s1] = Dp.y;
        }
        if (it.y + 1 < nch) {   // a middle chunk: counted as finished for the tile's last chunk
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(cons_done + tile, 1u);
            return;
        }
        // the tile's last chunk combines: its other consumers were all taken before it, so the bounded
        // wait ends; per pixel the colour is the sum of the chunks in chunk order, T_final and the last
        // contributor come from the last chunk whose walk ran (a chunk with T_in below t_min did not)
        if (threadIdx.x == 0) wait_geq(cons_done + tile, (uint32_t)(nch - 2), QUEUE_SPIN_LIMIT, flags);
        __syncthreads();
        const DevCam& cam = *g.cam;
        const int64_t plane = (int64_t)cam.width * cam.height;
        const float* E = exposure ? exposure + 12 * (g.cam - cams) : nullptr;
        const int64_t i0 = tile_item0[tile];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!(k ? g.in1 : g.in0)) continue;
            const int slot = k ? g.slot1 : g.slot0;
            const int py = k ? g.py_i1 : g.py_i0;
            float c0s = 0.0f, c1s = 0.0f, c2s = 0.0f, Ds = 0.0f, Tt = 1.0f, Tin = 1.0f;
            int lst = 0;
#pragma unroll 8
            for (int c = 0; c < nch; ++c) {
                const int64_t sl = (i0 + c) * NT + slot;
                const float c0 = __ldcg(sc.C + 3 * sl + 0), c1 = __ldcg(sc.C + 3 * sl + 1), c2 = __ldcg(sc.C + 3 * sl + 2);
                const float te = __ldcg(sc.Tend + sl), tc = __ldcg(sc.Tc + sl);   // Tc of the last chunk is not used
                const bool run = !(Tin < o.t_min);
                c0s += run ? c0 : 0.0f;
                c1s += run ? c1 : 0.0f;
                c2s += run ? c2 : 0.0f;
                Tt = run ? te : Tt;
                if (DEPTH) {
                    const float dd = __ldcg(sc.D + sl);
                    Ds += run ? dd : 0.0f;
                }
                if (SAVE) {
                    const int32_t l = __ldcg(sc.last + sl);
                    if (run && l >= 0) lst = l;
                }
                if (c + 1 < nch) Tin = fmul(Tin, tc);
            }
            const int64_t pix = cam.pix_base + (int64_t)py * cam.width + g.px_i;
            write_pixel(images + 3 * cam.pix_base + (int64_t)py * cam.width + g.px_i, plane, Tt, c0s, c1s, c2s, o, E);
            if (DEPTH) depth[pix] = Ds;
            if (SAVE) {
                T_final[pix] = Tt;
                n_contrib[pix] = lst;
            }
        }
        return;
    }
    const DevCam& cam = *g.cam;
    const int64_t plane = (int64_t)cam.width * cam.height;
    const float* E = exposure ? exposure + 12 * (g.cam - cams) : nullptr;
    if (g.in0) {
        const int64_t pix = cam.pix_base + (int64_t)g.py_i0 * cam.width + g.px_i;
        write_pixel(images + 3 * cam.pix_base + (int64_t)g.py_i0 * cam.width + g.px_i, plane, T.x, C0.x, C1.x, C2.x, o, E);
        if (DEPTH) depth[pix] = Dp.x;
        if (SAVE) {
            T_final[pix] = T.x;
            n_contrib[pix] = last.x < 0 ? 0 : last.x;
        }
    }
    if (g.in1) {
        const int64_t pix = cam.pix_base + (int64_t)g.py_i1 * cam.width + g.px_i;
        write_pixel(images + 3 * cam.pix_base + (int64_t)g.py_i1 * cam.width + g.px_i, plane, T.y, C0.y, C1.y, C2.y, o, E);
        if (DEPTH) depth[pix] = Dp.y;
        if (SAVE) {
            T_final[pix] = T.y;
            n_contrib[pix] = last.y < 0 ? 0 : last.y;
        }
    }
}

__global__ void wait_probe_kernel(const uint32_t* word, int polls, uint32_t* flags) {
    if (threadIdx.x == 0) wait_geq(word, 1u, polls, flags);
}

cudaError_t launch_wait_probe(const uint32_t* word, int polls, uint32_t* flags, cudaStream_t s) {
    wait_probe_kernel<<<1, 32, 0, s>>>(word, polls, flags);
    return cudaGetLastError();
}

size_t blend_plan_work_words(int64_t n_tiles) {
    return LB_HEADER_WORDS + 2 * (size_t)std::max<int64_t>(1, (n_tiles + PL_TILE - 1) / PL_TILE);
}

cudaError_t launch_blend(const BlendArgs& a, cudaStream_t s) {
    if (a.n_tiles <= 0) return cudaSuccess;
    const int64_t pblocks = (a.n_tiles + PL_TILE - 1) / PL_TILE;
    if ((size_t)(LB_HEADER_WORDS + 2 * pblocks) > a.work_words) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    if (!a.pre_zeroed) e = cudaMemsetAsync(a.work, 0, sizeof(uint32_t) * (LB_HEADER_WORDS + 2 * (size_t)pblocks), s);
    if (e != cudaSuccess) return e;
    Lookback lb{reinterpret_cast<unsigned long long*>(a.work + LB_HEADER_WORDS), a.work, a.flags};
    e = launch_dependent(blend_plan_kernel, dim3((unsigned)pblocks), dim3(PL_THREADS), s, a.ranges, a.n_tiles, a.chunk,
                         a.n_pairs, a.tile_item0, a.tile_nch, a.items, a.item_cap, a.q_prod, a.q_single, a.q_cons,
                         a.n_items, lb);
    if (e != cudaSuccess) return e;
    Scratch sc{a.scratch_Tc, a.scratch_C, a.scratch_Tend, a.scratch_last, a.scratch_D};
    if (!a.pre_zeroed) e = cudaMemsetAsync(a.queue_sync, 0, sizeof(uint32_t) * (size_t)(2 * a.n_tiles + 1), s);
    if (e != cudaSuccess) return e;
    // queue length 2 X + Y <= 2 item_cap - n_tiles
    const unsigned gq = (unsigned)std::max<int64_t>(1, 2 * a.item_cap - a.n_tiles);
#define QUEUE(TWV, THV, CNT, DEP, SAV)                                                                                \
    e = launch_dependent(blend_queue_kernel<TWV, THV, CNT, DEP, SAV>, dim3(gq), dim3(TWV * THV / 2), s,                \
        a.cams, a.n_cams, a.o, a.ranges, a.list, a.splat, a.n_splats, a.items, a.q_prod, a.q_single, a.q_cons,        \
        a.n_items,                                                                                                    \
        a.tile_item0, a.tile_nch, sc, a.queue_sync, a.queue_sync + 1, a.queue_sync + 1 + a.n_tiles, a.images,        \
        a.depth, a.exposure,                                                                                          \
        a.T_final, a.n_contrib, a.n_evals, a.flags)
#define BL(TWV, THV)                                                                                                  \
    do {                                                                                                              \
        if (a.ev_queue) cudaEventRecord(a.ev_queue[0], s);                                                            \
        if (a.depth) {                                                                                                \
            if (save) QUEUE(TWV, THV, false, true, true); else QUEUE(TWV, THV, false, true, false);                   \
        } else if (a.n_evals) {                                                                                       \
            if (save) QUEUE(TWV, THV, true, false, true); else QUEUE(TWV, THV, true, false, false);                   \
        } else {                                                                                                      \
            if (save) QUEUE(TWV, THV, false, false, true); else QUEUE(TWV, THV, false, false, false);                 \
        }                                                                                                             \
        if (e != cudaSuccess) break;                                                                                  \
        if (a.ev_queue) cudaEventRecord(a.ev_queue[1], s);                                                            \
    } while (0)
    const DevOpts& o = a.o;
    const bool save = a.T_final && a.n_contrib;   // per-pixel state for the adjoint (evaluations are not
                                                  // counted together with the depth output)
    if (o.tile_w == 16 && o.tile_h == 16) BL(16, 16);
    else if (o.tile_w == 8 && o.tile_h == 8) BL(8, 8);
    else if (o.tile_w == 32 && o.tile_h == 8) BL(32, 8);
    else if (o.tile_w == 8 && o.tile_h == 32) BL(8, 32);
    else if (o.tile_w == 16 && o.tile_h == 8) BL(16, 8);
    else return cudaErrorInvalidValue;
#undef BL
#undef QUEUE
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

H3DGS_CHECK_READER(check_read_blend)

}  // namespace h3dgs
