// Adjoint of the render path (a8), used to optimise interior hierarchy nodes (Sec. 5.1).
//
// Stage 1, per tile (one CTA, one thread per pixel): walk the tile's list back to front from the
// last contributor, recomputing each alpha exactly as the forward pass did (same fp32 decisions)
// and recovering the transmittance before each splat as T / (1 - alpha) from the saved final T, so
// nothing per (pixel, splat) is stored.  Per splat, the gradient w.r.t. its screen parameters
// (u, v, conic, o_n', o_p', colour) is summed over the warp with shuffles and added to a per-splat
// accumulator with one atomic per value per warp.  The alpha' chain uses the derivative of
// Eq. alphap, d alpha'/d alpha_p = (1/K)(1 - alpha_p)^(1/K - 1); an opacity gradient is zero on a
// clamped branch (Sec. 7.3).
//
// Stage 2, per cut entry: recompute the interpolated Gaussian and its projection and apply the
// adjoint of SH colour, EWA projection (Sigma' = M M^T, M = J W R(q) diag(s)), the opacity
// compensation and the quaternion normalisation, then scatter (1 - t) of the result to node n and
// t to its parent p (t is a constant; Sec. 5.1).  Leaves are skipped when frozen (Sec. 7.1).
#include "internal.cuh"

namespace h3dgs {

namespace {

constexpr float KH = -0.72134752044448170f;
constexpr float KL = 1.44269504088896341f;
constexpr float LN2 = 0.69314718055994531f;

constexpr float SH_C0 = 0.28209479177387814f;
constexpr float SH_C1 = 0.48860251190291992f;
constexpr float SH_C2A = 1.0925484305920792f;
constexpr float SH_C2B = 0.31539156525252005f;
constexpr float SH_C2C = 0.54627421529603959f;
constexpr float SH_C3A = 0.59004358992664352f;
constexpr float SH_C3B = 2.8906114426405538f;
constexpr float SH_C3C = 0.45704579946446572f;
constexpr float SH_C3D = 0.37317633259011540f;
constexpr float SH_C3E = 1.4453057213202769f;

__device__ __forceinline__ float alpha_prime_grad(float ap, float K) {
    if (K == 2.0f) return 0.5f * rsqrtf(1.0f - ap);
    return __fdividef(ex2_approx(lg2_approx(1.0f - ap) * (__fdividef(1.0f, K) - 1.0f)), K);
}

// Warp reduce-scatter of the per-lane gradient values of one splat: NV = 10 values (NV = 11 is done
// as 12 with a zero).  Each level halves the values a lane carries by exchanging half of them with
// the partner lane and adding; values left over at an odd count are reduced whole.  Afterwards the
// warp-wide sum of value k is in the lane returned by the caller's write step: *k_out is the value
// this lane writes (-1: none).  10 values: 14 shuffles; 12 values: 15.
template <int NV>
__device__ __forceinline__ float warp_reduce_scatter(const float* v, int lane, int* k_out) {
    const int b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1;
    auto xchg = [&](float lo, float hi, int off, bool upper) {
        const float send = upper ? lo : hi, keep = upper ? hi : lo;
        return keep + __shfl_xor_sync(0xffffffffu, send, off);
    };
    float y0, y1;
    if (NV == 10) {
        float w[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) w[i] = xchg(v[i], v[5 + i], 16, b4);   // value 5 b4 + i
        const float x0 = xchg(w[0], w[2], 8, b3);                           // 5 b4 + 2 b3
        const float x1 = xchg(w[1], w[3], 8, b3);                           // 5 b4 + 2 b3 + 1
        const float x2 = w[4] + __shfl_xor_sync(0xffffffffu, w[4], 8);      // 5 b4 + 4
        y0 = xchg(x0, x1, 4, b2);                                           // 5 b4 + 2 b3 + b2
        y1 = x2 + __shfl_xor_sync(0xffffffffu, x2, 4);
    } else {
        float w[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) w[i] = xchg(v[i], i + 6 < NV ? v[6 + i] : 0.0f, 16, b4);   // 6 b4 + i
        float x[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) x[i] = xchg(w[i], w[3 + i], 8, b3);     // 6 b4 + 3 b3 + i
        y0 = xchg(x[0], x[1], 4, b2);                                       // 6 b4 + 3 b3 + b2
        y1 = x[2] + __shfl_xor_sync(0xffffffffu, x[2], 4);                  // 6 b4 + 3 b3 + 2
    }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
    int k = -1;
    float val = 0.0f;
    if (NV == 10) {
        if ((lane & 3) == 0) { k = 5 * b4 + 2 * b3 + b2; val = y0; }
        else if ((lane & 15) == 1) { k = 5 * b4 + 4; val = y1; }
    } else {
        if ((lane & 3) == 0) { k = 6 * b4 + 3 * b3 + b2; val = y0; }
        else if ((lane & 7) == 1) { k = 6 * b4 + 3 * b3 + 2; val = y1; }
    }
    *k_out = k < NV ? k : -1;
    return val;
}

}  // namespace

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sel2(bool p0, bool p1, float2 a, float2 b) {
    return make_float2(p0 ? a.x : b.x, p1 ? a.y : b.y);
}

// One CTA per blend item (tile, chunk), TW x TH / 2 threads with two pixels each (the forward's
// layout: warp w owns an 8x8 block, lane l the pixels (l % 8, l / 8) and (l % 8, l / 8 + 4)).  A
// single-chunk tile starts from the pixel's final T and contributor count; a chunk of a split tile
// starts from the T at its end and its last contributor (saved by the forward pass), with the colour
// behind it = later chunks' colour + T_final bg.  Per splat the two pixels' gradients are added in
// registers before the warp reduction, and the arithmetic runs on pixel pairs.  The incoming
// gradient is taken back through the camera's exposure affine (dL/dC = E^T dL/dout); DEPTH adds the
// expected-depth channel (gradient dLdepth, the splat's view depth as its colour, no background).
template <int TW, int TH, bool DEPTH>
__global__ void __launch_bounds__(TW * TH / 2) backward_blend_kernel(const DevCam* __restrict__ cams, int n_cams,
                                                                     DevOpts o, const int2* __restrict__ ranges,
                                                                     const uint32_t* __restrict__ list,
                                                                     const float4* __restrict__ splat,
                                                                     const uint32_t* __restrict__ n_spl,
                                                                     const int2* __restrict__ items,
                                                                     const uint32_t* __restrict__ n_items,
                                                                     const int32_t* __restrict__ tile_item0,
                                                                     const int32_t* __restrict__ tile_nch,
                                                                     const float* __restrict__ scC,
                                                                     const float* __restrict__ scTend,
                                                                     const int32_t* __restrict__ sclast,
                                                                     const float* __restrict__ T_final,
                                                                     const int32_t* __restrict__ n_contrib,
                                                                     const float* __restrict__ dL,
                                                                     const float* __restrict__ dLdepth,
                                                                     const float* __restrict__ exposure,
                                                                     const float* __restrict__ scD,
                                                                     float* __restrict__ sgrad) {
    constexpr int NT = TW * TH, NT2 = NT / 2;
    __shared__ float4 s_a[NT2], s_b[NT2], s_c[NT2];
    __shared__ uint32_t s_id[NT2], s_m[NT2];
    __shared__ float s_dz[DEPTH ? NT2 : 1];
    __shared__ float4 s_box[NT2 / 32];
    __shared__ int s_max;
    const uint32_t item = blockIdx.x;
    if (item >= *n_items) return;
    const int2 it = items[item];
    const int64_t tile = it.x;
    const int nch = tile_nch[tile];
    int lo = 0, hi = n_cams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cams[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    const DevCam& cam = cams[lo];
    const int local = (int)(tile - cam.tile_base);
    const int ox = (local % cam.tiles_x) * TW, oy = (local / cam.tiles_x) * TH;
    int lx, ly0;
    tile_pixel2<TW, TH>(threadIdx.x, lx, ly0);
    const int px_i = ox + lx;
    const int pyi[2] = {oy + ly0, oy + ly0 + 4};
    const int lyk[2] = {ly0, ly0 + 4};
    const bool in_[2] = {px_i < cam.width && pyi[0] < cam.height, px_i < cam.width && pyi[1] < cam.height};
    const float px = (float)px_i + 0.5f;
    const float2 py = make_float2((float)pyi[0] + 0.5f, (float)pyi[1] + 0.5f);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 r = ranges[tile];
    const int begin = chunk_begin(r, nch, it.y);   // first list entry of this item
    float Tk[2] = {1.0f, 1.0f}, gk[2][3] = {{0, 0, 0}, {0, 0, 0}}, Sk[2][3] = {{0, 0, 0}, {0, 0, 0}};
    float gdk[2] = {0.0f, 0.0f}, SDk[2] = {0.0f, 0.0f};
    int stop[2] = {begin, begin};             // entries [begin, stop) are walked back to front
    const int64_t plane = (int64_t)cam.width * cam.height;
    const float* E = exposure ? exposure + 12 * lo : nullptr;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (!in_[k]) continue;
        const int64_t pix = cam.pix_base + (int64_t)pyi[k] * cam.width + px_i;
        const float* gp = dL + 3 * cam.pix_base + (int64_t)pyi[k] * cam.width + px_i;
        const float go0 = gp[0], go1 = gp[plane], go2 = gp[2 * plane];
        if (E) {
            for (int ch = 0; ch < 3; ++ch) gk[k][ch] = fmaf(E[ch], go0, fmaf(E[4 + ch], go1, E[8 + ch] * go2));
        } else {
            gk[k][0] = go0; gk[k][1] = go1; gk[k][2] = go2;
        }
        if (DEPTH) gdk[k] = dLdepth[pix];
        const float Tf = T_final[pix];
        for (int ch = 0; ch < 3; ++ch) Sk[k][ch] = Tf * o.bg[ch];
        if (nch == 1) {
            Tk[k] = Tf;
            stop[k] = r.x + n_contrib[pix];
        } else {
            const int64_t i0 = tile_item0[tile];
            const int64_t slot = (int64_t)item * NT + lyk[k] * TW + lx;   // the scratch is row-major per tile
            Tk[k] = scTend[slot];
            const int l = sclast[slot];
            stop[k] = l < 0 ? begin : r.x + l;
            for (int c = it.y + 1; c < nch; ++c) {
                const int64_t sl = (i0 + c) * NT + lyk[k] * TW + lx;
                for (int ch = 0; ch < 3; ++ch) Sk[k][ch] += scC[3 * sl + ch];
                if (DEPTH) SDk[k] += scD[sl];
            }
        }
    }
    float2 T = make_float2(Tk[0], Tk[1]);
    const float2 g0 = make_float2(gk[0][0], gk[1][0]), g1 = make_float2(gk[0][1], gk[1][1]),
                 g2 = make_float2(gk[0][2], gk[1][2]);
    const float2 S0 = make_float2(Sk[0][0], Sk[1][0]), S1 = make_float2(Sk[0][1], Sk[1][1]),
                 S2 = make_float2(Sk[0][2], Sk[1][2]);
    const float2 gd2 = make_float2(gdk[0], gdk[1]);
    // B = sum_c g_c S_c (+ g_depth S_depth): the colour behind the current splat, S_c, enters the alpha
    // adjoint only through this sum, which is carried instead of the channels
    float2 B = fma2(g2, S2, fma2(g1, S1, mul2(g0, S0)));
    if (DEPTH) B = fma2(gd2, make_float2(SDk[0], SDk[1]), B);
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    atomicMax(&s_max, max(stop[0], stop[1]) - begin);
    __syncthreads();
    const int count = s_max;
    const int last0 = stop[0] - begin, last1 = stop[1] - begin;
    const float clampv = o.alpha_clamp, afloor = o.alpha_floor;
    for (int end = count; end > 0; end -= NT2) {
        const int n = min(NT2, end);
        const int first = end - n;
        // bounding box of the warp's pixels that take part in this batch (their last contributor lies
        // beyond its first entry): the warp mask tests entries against it
        {
            const bool l0 = last0 > first, l1 = last1 > first, any_l = l0 || l1;
            const int iy_lo = l0 ? pyi[0] : pyi[1], iy_hi = l1 ? pyi[1] : pyi[0];
            const int xmin = __reduce_min_sync(0xffffffffu, any_l ? px_i : 0x7fffffff);
            const int xmax = __reduce_max_sync(0xffffffffu, any_l ? px_i : -1);
            const int ymin = __reduce_min_sync(0xffffffffu, any_l ? iy_lo : 0x7fffffff);
            const int ymax = __reduce_max_sync(0xffffffffu, any_l ? iy_hi : -1);
            if (lane == 0)
                s_box[warp] = xmax < 0 ? make_float4(1.0f, 1.0f, -1.0f, -1.0f)
                                       : make_float4((float)xmin + 0.5f, (float)ymin + 0.5f, (float)xmax + 0.5f,
                                                     (float)ymax + 0.5f);
        }
        __syncthreads();
        if ((int)threadIdx.x < n) {
            uint32_t s = __ldg(list + begin + first + threadIdx.x);
            if (!H3DGS_IN(s, *n_spl)) s = 0;   // checked build only
            const float4 a = __ldg(splat + SPLAT_F4 * (int64_t)s);
            const float4 d = __ldg(splat + SPLAT_F4 * (int64_t)s + 3);
            s_id[threadIdx.x] = s;
            s_a[threadIdx.x] = a;
            const float4 bb = __ldg(splat + SPLAT_F4 * (int64_t)s + 1);
            s_b[threadIdx.x] = bb;
            s_c[threadIdx.x] = __ldg(splat + SPLAT_F4 * (int64_t)s + 2);
            uint32_t wm = 0;
#pragma unroll
            for (int w = 0; w < NT2 / 32; ++w) {
                const float4 bx = s_box[w];
                if (bx.x <= bx.z && rect_reach(a, bb.x, d, bx.x, bx.y, bx.z, bx.w)) wm |= 1u << w;
            }
            s_m[threadIdx.x] = wm;
            if (DEPTH) s_dz[threadIdx.x] = d.w;
        }
        __syncthreads();
        // back to front over the splats that reach this warp's pixels
        for (int base = ((n - 1) >> 5) << 5; base >= 0; base -= 32) {
          const uint32_t mm = (base + lane < n) ? s_m[base + lane] : 0u;
          uint32_t bits = __ballot_sync(0xffffffffu, (mm >> warp) & 1u);
          while (bits) {
            const int hb = 31 - __clz(bits);
            bits &= ~(1u << hb);
            const int j = base + hb;
            const int pos = first + j;
            const bool act0 = pos < last0, act1 = pos < last1;
            if (!__any_sync(0xffffffffu, act0 || act1)) continue;
            const float4 a = s_a[j], b = s_b[j], c = s_c[j];
            // alpha exactly as the forward pass computed it (same fp32 order, paired per element)
            const float dx = fsub(px, a.x);
            const float2 dy = add2(py, f2(-a.y));
            const float2 h = fma2(f2(a.z), f2(dx), mul2(f2(a.w), dy));
            const float2 gq = mul2(mul2(f2(b.x), dy), dy);
            const float2 p2 = fma2(f2(dx), h, gq);
            const float2 G = make_float2(ex2_approx(p2.x), ex2_approx(p2.y));
            const float2 xn = mul2(f2(b.y), G);
            const float2 an = make_float2(fminf(clampv, xn.x), fminf(clampv, xn.y));
            float2 alpha = an, ap = f2(0.0f), xp = f2(0.0f);
            const bool interp = b.w != 0.0f;   // uniform over the warp
            if (interp) {
                xp = mul2(f2(b.z), G);
                ap = make_float2(fminf(clampv, xp.x), fminf(clampv, xp.y));
                const float omw = fsub(1.0f, b.w);
                alpha = fma2(f2(b.w), make_float2(alpha_prime(ap.x, c.w), alpha_prime(ap.y, c.w)), mul2(f2(omw), an));
            }
            const bool con0 = act0 && alpha.x >= afloor, con1 = act1 && alpha.y >= afloor;
            if (!__any_sync(0xffffffffu, con0 || con1)) continue;
            // one approximate reciprocal per pixel instead of four divisions (values, not decisions)
            const float2 inv = make_float2(__fdividef(1.0f, 1.0f - alpha.x), __fdividef(1.0f, 1.0f - alpha.y));
            T = sel2(con0, con1, mul2(T, inv), T);
            // a pixel that does not take the splat gets weight 0 and alpha adjoint 0, so every gradient
            // term below (each a product of one of the two with finite factors) is exactly 0 for it
            const float2 wgt = sel2(con0, con1, mul2(alpha, T), f2(0.0f));
            const float2 gr = mul2(g0, wgt), gg = mul2(g1, wgt), gb = mul2(g2, wgt);
            // alpha adjoint, colour part: sum_c g_c (T col_c - S_c / (1 - alpha)) = T A - B / (1 - alpha)
            float2 A = fma2(g2, f2(c.z), fma2(g1, f2(c.y), mul2(g0, f2(c.x))));
            float2 gz = f2(0.0f);
            if (DEPTH) {
                A = fma2(gd2, f2(s_dz[j]), A);
                gz = mul2(gd2, wgt);
            }
            float2 dal = fma2(T, A, mul2(B, mul2(inv, f2(-1.0f))));
            B = fma2(A, wgt, B);   // unchanged where wgt = 0
            dal = sel2(con0, con1, dal, f2(0.0f));
            const float2 dan = interp ? mul2(f2(1.0f - b.w), dal) : dal;
            const bool nl0 = xn.x < clampv, nl1 = xn.y < clampv;
            const float2 gon = sel2(nl0, nl1, mul2(dan, G), f2(0.0f));
            float2 dG = sel2(nl0, nl1, mul2(dan, f2(b.y)), f2(0.0f));
            float2 gop = f2(0.0f);
            if (interp) {
                const bool pl0 = xp.x < clampv, pl1 = xp.y < clampv;
                const float2 dap = mul2(mul2(f2(b.w), dal),
                                        make_float2(alpha_prime_grad(ap.x, c.w), alpha_prime_grad(ap.y, c.w)));
                gop = sel2(pl0, pl1, mul2(dap, G), f2(0.0f));
                dG = sel2(pl0, pl1, fma2(dap, f2(b.z), dG), dG);
            }
            const float2 dp2 = mul2(mul2(dG, G), f2(LN2));
            // exponent p2 = ca dx^2 + cb dx dy + cc dy^2 with dx = px - u, dy = py - v: the conic gradients
            // are dp2 dx^2, dp2 dx dy, dp2 dy^2, and the mean gradients -(2 ca P + cb Q), -(cb P + 2 cc Q)
            // are linear in P = sum dp2 dx and Q = sum dp2 dy, which are reduced instead (the splat stage
            // applies the conic once per splat)
            const float2 P = mul2(dp2, f2(dx)), Q = mul2(dp2, dy);
            const float2 gca = mul2(P, f2(dx)), gcb = mul2(P, dy), gcc = mul2(Q, dy);
            // both pixels' contributions of this splat (a pixel that does not take it adds zero)
            auto sum2 = [](float2 x) { return x.x + x.y; };
            const float v[11] = {sum2(P), sum2(Q), sum2(gca), sum2(gcb), sum2(gcc), sum2(gon), sum2(gop), sum2(gr),
                                 sum2(gg), sum2(gb), DEPTH ? sum2(gz) : 0.f};
            int kk;
            const float sum = warp_reduce_scatter<DEPTH ? 11 : 10>(v, lane, &kk);
            if (kk >= 0) atomicAdd(sgrad + 12 * (int64_t)s_id[j] + kk, sum);
          }
        }
    }
}

// ---------------------------------------------------------------------------------------- stage 2

// Vector reduction of 4 floats (16-byte aligned address) into global memory.
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

__global__ void __launch_bounds__(128) backward_splat_kernel(DevHier h, const DevCam* __restrict__ cams, int n_cams,
                                                            DevOpts o, const int32_t* __restrict__ cut_ids,
                                                            const float* __restrict__ cut_t,
                                                            const int64_t* __restrict__ cut_offsets,
                                                            const uint2* __restrict__ rect,
                                                            const uint32_t* __restrict__ n_splats,
                                                            const float* __restrict__ sgrad, GradBufs gout,
                                                            int freeze_leaves) {
    const uint32_t M = *n_splats;
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        if (rect[m].x == 0xffffffffu) continue;  // culled
        const float* gs = sgrad + 12 * (int64_t)m;
        // gs: sum dp2 dx, sum dp2 dy, the three conic gradients, the two opacity gradients, colour, depth
        const float sP = gs[0], sQ = gs[1], gca = gs[2], gcb = gs[3], gcc = gs[4], gon = gs[5], gop = gs[6];
        const float gz = gs[10];   // expected-depth channel: d L / d (view depth of the mean)
        const float grgb[3] = {gs[7], gs[8], gs[9]};
        const int k = find_cam(cut_offsets, n_cams, m);
        const DevCam& cam = cams[k];
        const int32_t n = cut_ids[m];
        if (!H3DGS_IN(n, h.n)) continue;   // checked build only
        const float t = (o.interpolate && cut_t) ? cut_t[m] : 0.0f;
        const int32_t p = h.parent[n];
        const bool use_p = (t != 0.0f) && p >= 0 && H3DGS_IN(p, h.n);
        const float omt = 1.0f - t;
        // ---- interpolated attributes
        float s[3], ql[4];
        const float4 qn4 = h.rot[n];
        float qv[4] = {qn4.x, qn4.y, qn4.z, qn4.w};
        for (int d = 0; d < 3; ++d) s[d] = h.scale[3 * (int64_t)n + d];
        if (use_p) {
            const float4 qp4 = h.rot[p];
            const float qpv[4] = {qp4.x, qp4.y, qp4.z, qp4.w};
            for (int d = 0; d < 3; ++d) s[d] = fmaf(t, h.scale[3 * (int64_t)p + d], omt * s[d]);
            for (int d = 0; d < 4; ++d) qv[d] = fmaf(t, qpv[d], omt * qv[d]);
        }
        for (int d = 0; d < 4; ++d) ql[d] = qv[d];
        const float qnorm = sqrtf(ql[0] * ql[0] + ql[1] * ql[1] + ql[2] * ql[2] + ql[3] * ql[3]);
        const float q[4] = {ql[0] / qnorm, ql[1] / qnorm, ql[2] / qnorm, ql[3] / qnorm};
        // ---- forward recompute
        const float* W = cam.R;
        // the camera-space mean exactly as the forward pass formed it (compensated transforms of the
        // node's and the parent's means, interpolated in camera space)
        float xc[3];
        view_point(W, cam.T, h.mean[3 * (int64_t)n], h.mean[3 * (int64_t)n + 1], h.mean[3 * (int64_t)n + 2], xc);
        if (use_p) {
            float xp[3];
            view_point(W, cam.T, h.mean[3 * (int64_t)p], h.mean[3 * (int64_t)p + 1], h.mean[3 * (int64_t)p + 2], xp);
            for (int i = 0; i < 3; ++i) xc[i] = ffma(t, xp[i], fmul(fsub(1.0f, t), xc[i]));
        }
        const float z = xc[2], iz = 1.0f / z;
        const float xz = xc[0] * iz, yz = xc[1] * iz;
        const bool x_in = xz > -cam.limx && xz < cam.limx, y_in = yz > -cam.limy && yz < cam.limy;
        const float txc = fminf(fmaxf(xz, -cam.limx), cam.limx), tyc = fminf(fmaxf(yz, -cam.limy), cam.limy);
        const float fx = cam.fx, fy = cam.fy;
        const float J00 = fx * iz, J02 = -fx * txc * iz, J11 = fy * iz, J12 = -fy * tyc * iz;
        float A2[2][3];
        for (int j = 0; j < 3; ++j) {
            A2[0][j] = J00 * W[j] + J02 * W[6 + j];
            A2[1][j] = J11 * W[3 + j] + J12 * W[6 + j];
        }
        const float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
        float Rq[3][3];
        Rq[0][0] = 1.f - 2.f * (qy * qy + qz * qz); Rq[0][1] = 2.f * (qx * qy - qw * qz); Rq[0][2] = 2.f * (qx * qz + qw * qy);
        Rq[1][0] = 2.f * (qx * qy + qw * qz); Rq[1][1] = 1.f - 2.f * (qx * qx + qz * qz); Rq[1][2] = 2.f * (qy * qz - qw * qx);
        Rq[2][0] = 2.f * (qx * qz - qw * qy); Rq[2][1] = 2.f * (qy * qz + qw * qx); Rq[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
        float B[2][3], M[2][3];
        for (int i = 0; i < 2; ++i)
            for (int kk = 0; kk < 3; ++kk) {
                B[i][kk] = A2[i][0] * Rq[0][kk] + A2[i][1] * Rq[1][kk] + A2[i][2] * Rq[2][kk];
                M[i][kk] = B[i][kk] * s[kk];
            }
        const float aa = M[0][0] * M[0][0] + M[0][1] * M[0][1] + M[0][2] * M[0][2];
        const float cc = M[1][0] * M[1][0] + M[1][1] * M[1][1] + M[1][2] * M[1][2];
        const float bb = M[0][0] * M[1][0] + M[0][1] * M[1][1] + M[0][2] * M[1][2];
        const float k0 = M[0][1] * M[1][2] - M[0][2] * M[1][1];
        const float k1 = M[0][2] * M[1][0] - M[0][0] * M[1][2];
        const float k2 = M[0][0] * M[1][1] - M[0][1] * M[1][0];
        const float det = k0 * k0 + k1 * k1 + k2 * k2;
        const float lp = o.lowpass;
        const float af = aa + lp, cf = cc + lp;
        const float D = det + lp * (aa + cc + lp);
        const float iD = 1.0f / D;
        const float comp = o.aa_compensate ? sqrtf(fmaxf(0.0f, det * iD)) : 1.0f;
        const float ca = cf * iD * KH, cb = bb * iD * KL, cq = af * iD * KH;
        // mean (pixel-space) gradients from the reduced sums
        const float gu = -fmaf(2.0f * ca, sP, cb * sQ), gv = -fmaf(cb, sP, 2.0f * cq * sQ);
        // ---- opacities
        const float on = h.opacity[n], op = use_p ? h.opacity[p] : 0.0f;
        const float d_on = gon * comp, d_op = gop * comp;
        const float dcomp = gon * on + gop * op;
        // ---- conic -> (aa, bb, cc)
        float dD = -(gca * ca + gcb * cb + gcc * cq) * iD;
        float dcf = gca * KH * iD, daf = gcc * KH * iD, dbb = gcb * KL * iD;
        float ddet = 0.0f;
        if (o.aa_compensate && comp > 0.0f) {
            ddet = dcomp / (2.0f * comp * D);
            dD += -dcomp * comp / (2.0f * D);
        }
        daf += dD * cf; dcf += dD * af; dbb += dD * (-2.0f * bb);
        const float daa = daf + ddet * cc, dcc = dcf + ddet * aa;
        dbb += ddet * (-2.0f * bb);
        float dM[2][3], dB[2][3], ds[3];
        for (int kk = 0; kk < 3; ++kk) {
            dM[0][kk] = 2.0f * daa * M[0][kk] + dbb * M[1][kk];
            dM[1][kk] = 2.0f * dcc * M[1][kk] + dbb * M[0][kk];
            ds[kk] = dM[0][kk] * B[0][kk] + dM[1][kk] * B[1][kk];
            dB[0][kk] = dM[0][kk] * s[kk];
            dB[1][kk] = dM[1][kk] * s[kk];
        }
        float dRq[3][3], dA2[2][3];
        for (int j = 0; j < 3; ++j)
            for (int kk = 0; kk < 3; ++kk) dRq[j][kk] = A2[0][j] * dB[0][kk] + A2[1][j] * dB[1][kk];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) dA2[i][j] = dB[i][0] * Rq[j][0] + dB[i][1] * Rq[j][1] + dB[i][2] * Rq[j][2];
        const float dJ00 = dA2[0][0] * W[0] + dA2[0][1] * W[1] + dA2[0][2] * W[2];
        const float dJ02 = dA2[0][0] * W[6] + dA2[0][1] * W[7] + dA2[0][2] * W[8];
        const float dJ11 = dA2[1][0] * W[3] + dA2[1][1] * W[4] + dA2[1][2] * W[5];
        const float dJ12 = dA2[1][0] * W[6] + dA2[1][1] * W[7] + dA2[1][2] * W[8];
        const float iz2 = iz * iz;
        float dz = -dJ00 * fx * iz2 + dJ02 * fx * txc * iz2 - dJ11 * fy * iz2 + dJ12 * fy * tyc * iz2;
        const float dtxc = -dJ02 * fx * iz, dtyc = -dJ12 * fy * iz;
        const float dxz = gu * fx + (x_in ? dtxc : 0.0f);
        const float dyz = gv * fy + (y_in ? dtyc : 0.0f);
        const float dxc[3] = {dxz * iz, dyz * iz, dz + gz - dxz * xc[0] * iz2 - dyz * xc[1] * iz2};
        float dmu[3];
        for (int j = 0; j < 3; ++j) dmu[j] = W[j] * dxc[0] + W[3 + j] * dxc[1] + W[6 + j] * dxc[2];
        // rotation matrix w.r.t. the unit quaternion
        float dq[4];
        dq[0] = 2.f * (-qz * dRq[0][1] + qy * dRq[0][2] + qz * dRq[1][0] - qx * dRq[1][2] - qy * dRq[2][0] + qx * dRq[2][1]);
        dq[1] = 2.f * (qy * dRq[0][1] + qz * dRq[0][2] + qy * dRq[1][0] - 2.f * qx * dRq[1][1] - qw * dRq[1][2] +
                       qz * dRq[2][0] + qw * dRq[2][1] - 2.f * qx * dRq[2][2]);
        dq[2] = 2.f * (-2.f * qy * dRq[0][0] + qx * dRq[0][1] + qw * dRq[0][2] + qx * dRq[1][0] + qz * dRq[1][2] -
                       qw * dRq[2][0] + qz * dRq[2][1] - 2.f * qy * dRq[2][2]);
        dq[3] = 2.f * (-2.f * qz * dRq[0][0] - qw * dRq[0][1] + qx * dRq[0][2] + qw * dRq[1][0] - 2.f * qz * dRq[1][1] +
                       qy * dRq[1][2] + qx * dRq[2][0] + qy * dRq[2][1]);
        const float qdot = q[0] * dq[0] + q[1] * dq[1] + q[2] * dq[2] + q[3] * dq[3];
        float dql[4];
        for (int d = 0; d < 4; ++d) dql[d] = (dq[d] - q[d] * qdot) / qnorm;
        // ---- colour
        // view direction mean - c, as in the forward pass
        float dv[3];
        for (int j = 0; j < 3; ++j) {
            const float dn = (h.mean[3 * (int64_t)n + j] - cam.ch[j]) - cam.cl[j];
            dv[j] = use_p ? fmaf(t, (h.mean[3 * (int64_t)p + j] - cam.ch[j]) - cam.cl[j], omt * dn) : dn;
        }
        const float dn = sqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        const float x = dv[0] / dn, y = dv[1] / dn, zz = dv[2] / dn;
        const float xx = x * x, yy = y * y, z2 = zz * zz;
        float Y[16];
        Y[0] = SH_C0;
        Y[1] = -SH_C1 * y; Y[2] = SH_C1 * zz; Y[3] = -SH_C1 * x;
        Y[4] = SH_C2A * x * y; Y[5] = -SH_C2A * y * zz; Y[6] = SH_C2B * (2.f * z2 - xx - yy);
        Y[7] = -SH_C2A * x * zz; Y[8] = SH_C2C * (xx - yy);
        Y[9] = -SH_C3A * y * (3.f * xx - yy); Y[10] = SH_C3B * x * y * zz;
        Y[11] = -SH_C3C * y * (4.f * z2 - xx - yy); Y[12] = SH_C3D * zz * (2.f * z2 - 3.f * xx - 3.f * yy);
        Y[13] = -SH_C3C * x * (4.f * z2 - xx - yy); Y[14] = SH_C3E * zz * (xx - yy);
        Y[15] = -SH_C3A * x * (xx - 3.f * yy);
        // SH rows as float4 (12 per node); loops fully unrolled so every Y / dY index is a constant
        const float4* shn4 = h.sh + (int64_t)12 * n;
        const float4* shp4 = h.sh + (int64_t)12 * (use_p ? p : n);
        float col[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int j4 = 0; j4 < 12; ++j4) {
            const float4 a4 = __ldg(shn4 + j4);
            float4 v4 = a4;
            if (use_p) {
                const float4 b4 = __ldg(shp4 + j4);
                v4 = make_float4(fmaf(t, b4.x, omt * a4.x), fmaf(t, b4.y, omt * a4.y), fmaf(t, b4.z, omt * a4.z),
                                 fmaf(t, b4.w, omt * a4.w));
            }
            const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) col[(4 * j4 + e) % 3] += vv[e] * Y[(4 * j4 + e) / 3];
        }
        // wk[k] = sum over the channels that are not clamped of dL/dcolour x coefficient k (the colour's
        // derivative along the view direction is then sum_k wk[k] dY_k)
        float wk[16];
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) wk[kk] = 0.0f;
        const float wn = use_p ? omt : 1.0f;
        const bool leaf_n = h.child_count[n] == 0;
        const bool write_n = !(freeze_leaves && leaf_n);
        // SH gradient in groups of 4 coefficients, one vector reduction per group and row
#pragma unroll
        for (int j4 = 0; j4 < 12; ++j4) {
            const float4 a4 = __ldg(shn4 + j4);
            float4 v4 = a4;
            if (use_p) {
                const float4 b4 = __ldg(shp4 + j4);
                v4 = make_float4(fmaf(t, b4.x, omt * a4.x), fmaf(t, b4.y, omt * a4.y), fmaf(t, b4.z, omt * a4.z),
                                 fmaf(t, b4.w, omt * a4.w));
            }
            const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
            float g4[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 4 * j4 + e, ch = c % 3;
                const bool live = !(col[ch] < 0.0f);
                g4[e] = live ? grgb[ch] * Y[c / 3] : 0.0f;
                if (live) wk[c / 3] += grgb[ch] * vv[e];
            }
            if (g4[0] != 0.0f || g4[1] != 0.0f || g4[2] != 0.0f || g4[3] != 0.0f) {
                if (write_n) red_add_v4(gout.sh + (int64_t)NSH * n + 4 * j4, wn * g4[0], wn * g4[1], wn * g4[2], wn * g4[3]);
                if (use_p) red_add_v4(gout.sh + (int64_t)NSH * p + 4 * j4, t * g4[0], t * g4[1], t * g4[2], t * g4[3]);
            }
        }
        // derivatives of the basis functions along x, y, z (built after the coefficient loops, so they
        // are not held across them)
        float dY[16][3];
        for (int kk = 0; kk < 16; ++kk) dY[kk][0] = dY[kk][1] = dY[kk][2] = 0.f;
        dY[1][1] = -SH_C1; dY[2][2] = SH_C1; dY[3][0] = -SH_C1;
        dY[4][0] = SH_C2A * y; dY[4][1] = SH_C2A * x;
        dY[5][1] = -SH_C2A * zz; dY[5][2] = -SH_C2A * y;
        dY[6][0] = -2.f * SH_C2B * x; dY[6][1] = -2.f * SH_C2B * y; dY[6][2] = 4.f * SH_C2B * zz;
        dY[7][0] = -SH_C2A * zz; dY[7][2] = -SH_C2A * x;
        dY[8][0] = 2.f * SH_C2C * x; dY[8][1] = -2.f * SH_C2C * y;
        dY[9][0] = -6.f * SH_C3A * x * y; dY[9][1] = -SH_C3A * (3.f * xx - 3.f * yy);
        dY[10][0] = SH_C3B * y * zz; dY[10][1] = SH_C3B * x * zz; dY[10][2] = SH_C3B * x * y;
        dY[11][0] = 2.f * SH_C3C * x * y; dY[11][1] = -SH_C3C * (4.f * z2 - xx - 3.f * yy); dY[11][2] = -8.f * SH_C3C * y * zz;
        dY[12][0] = -6.f * SH_C3D * x * zz; dY[12][1] = -6.f * SH_C3D * y * zz; dY[12][2] = SH_C3D * (6.f * z2 - 3.f * xx - 3.f * yy);
        dY[13][0] = -SH_C3C * (4.f * z2 - 3.f * xx - yy); dY[13][1] = 2.f * SH_C3C * x * y; dY[13][2] = -8.f * SH_C3C * x * zz;
        dY[14][0] = 2.f * SH_C3E * zz * x; dY[14][1] = -2.f * SH_C3E * zz * y; dY[14][2] = SH_C3E * (xx - yy);
        dY[15][0] = -SH_C3A * (3.f * xx - 3.f * yy); dY[15][1] = 6.f * SH_C3A * x * y;
        float ddir[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 1; kk < 16; ++kk)
            for (int jj = 0; jj < 3; ++jj) ddir[jj] += wk[kk] * dY[kk][jj];
        const float dot = ddir[0] * x + ddir[1] * y + ddir[2] * zz;
        dmu[0] += (ddir[0] - x * dot) / dn;
        dmu[1] += (ddir[1] - y * dot) / dn;
        dmu[2] += (ddir[2] - zz * dot) / dn;
        // ---- scatter to node and parent
        if (write_n) {
            for (int d = 0; d < 3; ++d) {
                atomicAdd(gout.mean + 3 * (int64_t)n + d, wn * dmu[d]);
                atomicAdd(gout.scale + 3 * (int64_t)n + d, wn * ds[d]);
            }
            red_add_v4(gout.rot + 4 * (int64_t)n, wn * dql[0], wn * dql[1], wn * dql[2], wn * dql[3]);
            atomicAdd(gout.opacity + n, d_on);
        }
        if (use_p) {
            for (int d = 0; d < 3; ++d) {
                atomicAdd(gout.mean + 3 * (int64_t)p + d, t * dmu[d]);
                atomicAdd(gout.scale + 3 * (int64_t)p + d, t * ds[d]);
            }
            red_add_v4(gout.rot + 4 * (int64_t)p, t * dql[0], t * dql[1], t * dql[2], t * dql[3]);
            atomicAdd(gout.opacity + p, d_op);
        }
    }
}

cudaError_t launch_backward(const DevHier& h, const BlendArgs& a, const int32_t* cut_ids, const float* cut_t,
                            const int64_t* cut_offsets, const uint2* rect, const uint32_t* n_splats, const float* dL,
                            const float* dLdepth, float* splat_grad, const GradBufs& g, int freeze_leaves, int grid,
                            cudaEvent_t* ev, cudaStream_t s) {
    if (ev) cudaEventRecord(ev[0], s);
    if (a.n_tiles > 0) {
        const unsigned ig = (unsigned)a.item_cap;
#define BWD(TWV, THV, DEP)                                                                                          \
    backward_blend_kernel<TWV, THV, DEP><<<ig, TWV * THV / 2, 0, s>>>(                                              \
        a.cams, a.n_cams, a.o, a.ranges, a.list, a.splat, n_splats, a.items, a.n_items, a.tile_item0, a.tile_nch,     \
        a.scratch_C, a.scratch_Tend, a.scratch_last, a.T_final, a.n_contrib, dL, dLdepth, a.exposure, a.scratch_D,    \
        splat_grad)
#define BW(TWV, THV)                                                                                                \
    do {                                                                                                            \
        if (dLdepth) BWD(TWV, THV, true); else BWD(TWV, THV, false);                                                \
    } while (0)
        const DevOpts& o = a.o;
        if (o.tile_w == 16 && o.tile_h == 16) BW(16, 16);
        else if (o.tile_w == 8 && o.tile_h == 8) BW(8, 8);
        else if (o.tile_w == 32 && o.tile_h == 8) BW(32, 8);
        else if (o.tile_w == 8 && o.tile_h == 32) BW(8, 32);
        else if (o.tile_w == 16 && o.tile_h == 8) BW(16, 8);
        else return cudaErrorInvalidValue;
#undef BW
#undef BWD
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (ev) {
        cudaEventRecord(ev[1], s);
        cudaEventRecord(ev[2], s);
    }
    backward_splat_kernel<<<grid, 128, 0, s>>>(h, a.cams, a.n_cams, a.o, cut_ids, cut_t, cut_offsets, rect, n_splats,
                                               splat_grad, g, freeze_leaves);
    if (ev) cudaEventRecord(ev[3], s);
    return cudaGetLastError();
}

H3DGS_CHECK_READER(check_read_backward)

}  // namespace h3dgs
