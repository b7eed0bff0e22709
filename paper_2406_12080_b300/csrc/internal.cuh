// Internal declarations shared by the CUDA translation units of libh3dgs (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "h3dgs.h"

namespace h3dgs {

constexpr int NSH = 48;          // degree-3 SH: 16 basis functions x 3 channels, layout [k*3 + ch]
constexpr int NINTERP = 62;      // exported interpolated row: mean 3, scale 3, rot 4, sh 48, o_n, o_p, t, K
constexpr int MAX_CAMS = 4096;
constexpr int CAM_BATCH = 32;    // cameras per set-up launch (passed by value)
constexpr size_t LB_HEADER_WORDS = 64;   // look-back workspaces: ticket word(s), then 2 words per block

// Device flag bits (ctx->d_flags)
constexpr uint32_t FLAG_PAIRS_OVERFLOW = 1u << 0;
constexpr uint32_t FLAG_SPLATS_OVERFLOW = 1u << 1;
constexpr uint32_t FLAG_CUT_TRUNCATED = 1u << 2;
constexpr uint32_t FLAG_WAIT_TIMEOUT = 1u << 3;   // a bounded wait on another block gave up (frame invalid)
constexpr uint32_t FLAG_BAD_TOPOLOGY = 1u << 4;   // a parent index not below its child's (compaction)
constexpr uint32_t FLAG_NOT_RESIDENT = 1u << 5;   // streamed hierarchy: a cut node's attributes not in the cache
constexpr uint32_t FLAG_CACHE_FULL = 1u << 6;     // streamed hierarchy: too few free cache slots for an update
constexpr uint32_t FLAG_BOUNDS = 1u << 7;         // checked build: an index failed its bounds check

// ---------------------------------------------------------------- debug bounds checks
// A build with -DH3DGS_CHECK (paper_2406_12080_b300/build.py --check: libh3dgs_check.so) tests every
// index that comes from data -- a parent id, a cut id, a list entry, a staging slot or a scatter
// destination of the radix sort, a work item -- against the buffer it addresses before the access.  A
// failed check records the source line in its translation unit's check word and the access is
// skipped or redirected to element 0; a few invariants are tested the same way (H3DGS_HOLDS); nothing
// traps, so the context stays usable and the host reads
// the words (h3dgs_get_stats: FLAG_BOUNDS, and the file and line in h3dgs_last_error).  The default
// build compiles every check to `true`.
#ifdef H3DGS_CHECK
static __device__ uint32_t g_check_word[2];   // [0]: 1 once a check failed; [1]: the line of the first
__device__ __forceinline__ bool check_in(int64_t i, int64_t n, int line) {
    if (i >= 0 && i < n) return true;
    if (atomicCAS(&g_check_word[0], 0u, 1u) == 0u) atomicExch(&g_check_word[1], (uint32_t)line);
    return false;
}
#define H3DGS_IN(i, n) ::h3dgs::check_in((int64_t)(i), (int64_t)(n), __LINE__)
// an invariant that the kernel relies on (recorded like a failed range check)
#define H3DGS_HOLDS(c) ((void)::h3dgs::check_in((c) ? 0 : -1, 1, __LINE__))
#define H3DGS_CHECK_READER(name)                                                                              \
    cudaError_t name(uint32_t out[2], cudaStream_t s) {                                                         \
        cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_check_word, sizeof(uint32_t) * 2, 0,                  \
                                                  cudaMemcpyDeviceToHost, s);                                    \
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);                                                     \
        const uint32_t zero[2] = {0u, 0u};                                                                      \
        if (e == cudaSuccess && out[0])                                                                         \
            e = cudaMemcpyToSymbolAsync(g_check_word, zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s);        \
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);                                                     \
        return e;                                                                                               \
    }
#else
#define H3DGS_IN(i, n) true
#define H3DGS_HOLDS(c) ((void)0)
#define H3DGS_CHECK_READER(name)                                                                              \
    cudaError_t name(uint32_t out[2], cudaStream_t) {                                                           \
        out[0] = out[1] = 0u;                                                                                   \
        return cudaSuccess;                                                                                     \
    }
#endif
// The check words of the checked translation units: out[0] = 1 if a check failed since the last read
// (reading clears it), out[1] = the source line of the first failure.
cudaError_t check_read_cut(uint32_t out[2], cudaStream_t s);
cudaError_t check_read_preprocess(uint32_t out[2], cudaStream_t s);
cudaError_t check_read_sort(uint32_t out[2], cudaStream_t s);
cudaError_t check_read_blend(uint32_t out[2], cudaStream_t s);
cudaError_t check_read_backward(uint32_t out[2], cudaStream_t s);
constexpr int QUEUE_SPIN_LIMIT = 1 << 22;          // polls of the blend queue's per-tile counter

// Per-camera data on the device.  Raw fields come from h3dgs_camera; the derived floats are
// computed on the device in a fixed fp32 order (camera_setup kernel); integer bookkeeping
// (tile grid, offsets into the packed tile/pixel spaces) is filled on the host.
struct DevCam {
    float R[9];
    float T[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear, tau;
    float c[3];        // camera centre  -R^T T (fixed fp32 order: the granularity's decisions)
    float ch[3], cl[3];// the centre as an unevaluated sum ch + cl of a compensated dot product (values)
    float f;           // max(fx, fy)
    float limx, limy;  // 1.3 tan(half fov): clamp of x/z, y/z in the EWA Jacobian
    int32_t tiles_x, tiles_y;
    int64_t tile_base; // first global tile index of this camera
    int64_t pix_base;  // first pixel of this camera in the packed pixel space
};

struct CamBatch {
    int32_t first, count;
    h3dgs_camera cam[CAM_BATCH];
    int32_t tiles_x[CAM_BATCH], tiles_y[CAM_BATCH];
    int64_t tile_base[CAM_BATCH], pix_base[CAM_BATCH];
};

// Render options as used on the device.
struct DevOpts {
    int32_t tile_w, tile_h, chunk;
    float lowpass, alpha_clamp, alpha_floor, t_min;
    int32_t aa_compensate, interpolate;
    float bg[3];
};

// Borrowed hierarchy arrays (device).
struct DevHier {
    int64_t n;
    const float* mean;
    const float* scale;
    const float4* rot;
    const float* opacity;
    const float4* sh;      // [N][12] float4
    const int32_t* parent;
    const int32_t* child_count;
    const float4* rec;     // packed cut records [N][2]: {box_min.xyz, parent}, {box_max.xyz, child_count}
    const float4* row_bound;  // per row of 256 nodes of the one-camera scan [rows][2]: {parents' union box
                              // min, their largest side}, {union box max, 1 if the row is never skipped}, or NULL
    const int32_t* row_of; // attribute row of each node (streamed hierarchy: its cache slot, -1 if absent), or
                           // NULL: the node id
};

// ---------------------------------------------------------------- fp32 ops in a fixed order
// These never contract into FMA (and ffma always is one), so both sides of the parity tests can
// evaluate integer decisions bit-identically.
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// World -> camera transform of one point, x_c[i] = R_i . m + T_i, as a compensated dot product
// (Ogita, Rump & Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005: Dot2,
// with the products split exactly by an FMA and the sums by Knuth's TwoSum).  Large scenes keep
// their coordinates in metres over kilometres, where fp32 resolves about 3e-5 m, while a splat a
// metre in front of the camera needs camera-space coordinates far finer than that: the plain
// fmaf chain loses them to cancellation between R m and T (up to 0.05 px at 720p for near splats);
// Dot2 returns the point as if the dot product were evaluated in twice the working precision and
// then rounded.  Fixed fp32 order: products (R_i0 m_0), (R_i1 m_1), (R_i2 m_2), then T_i.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = fadd(a, b);
    const float z = fsub(s, a);
    e = fadd(fsub(a, fsub(s, z)), fsub(b, z));
}
// r0 m0 + r1 m1 + r2 m2 + b as the unevaluated sum hi + lo (Dot2 before its final addition)
__device__ __forceinline__ void dot2_pair(float r0, float r1, float r2, float b, float m0, float m1, float m2,
                                          float& hi, float& lo) {
    float p = fmul(r0, m0);
    float err = ffma(r0, m0, -p);
    const float rv[2] = {r1, r2}, mv[2] = {m1, m2};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float h = fmul(rv[j], mv[j]);
        const float r = ffma(rv[j], mv[j], -h);
        float q;
        two_sum(p, h, p, q);
        err = fadd(err, fadd(q, r));
    }
    float q;
    two_sum(p, b, p, q);
    hi = p;
    lo = fadd(err, q);
}
__device__ __forceinline__ float dot2_row(const float* Ri, float Ti, float m0, float m1, float m2) {
    float hi, lo;
    dot2_pair(Ri[0], Ri[1], Ri[2], Ti, m0, m1, m2, hi, lo);
    return fadd(hi, lo);
}
__device__ __forceinline__ void view_point(const float* R, const float* T, float m0, float m1, float m2, float xc[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) xc[i] = dot2_row(R + 3 * i, T[i], m0, m1, m2);
}

// Granularity (Sec. 4.2): projected size of the node's box, largest side over the distance from the
// camera centre to the closest point of the box; +inf with the camera inside the box.
// c = the camera centre, f = max(fx, fy).
__device__ __forceinline__ float granularity(float c0, float c1, float c2, float f, float lx, float ly, float lz,
                                             float hx, float hy, float hz) {
    const float dx = fmaxf(fmaxf(fsub(lx, c0), fsub(c0, hx)), 0.0f);
    const float dy = fmaxf(fmaxf(fsub(ly, c1), fsub(c1, hy)), 0.0f);
    const float dz = fmaxf(fmaxf(fsub(lz, c2), fsub(c2, hz)), 0.0f);
    float d2 = fmul(dx, dx);
    d2 = ffma(dy, dy, d2);
    d2 = ffma(dz, dz, d2);
    const float size = fmaxf(fmaxf(fsub(hx, lx), fsub(hy, ly)), fsub(hz, lz));
    if (d2 == 0.0f) return __int_as_float(0x7f800000);
    return fdiv(fmul(f, size), fsqrt(d2));
}
__device__ __forceinline__ float granularity(const DevCam& cam, float lx, float ly, float lz, float hx, float hy,
                                             float hz) {
    return granularity(cam.c[0], cam.c[1], cam.c[2], cam.f, lx, ly, lz, hx, hy, hz);
}

// Camera centre c = -R^T T, component j as -fmaf(R_2j, T_2, fmaf(R_1j, T_1, R_0j * T_0)).
__device__ __forceinline__ void camera_centre(const h3dgs_camera& cam, float c[3]) {
    for (int j = 0; j < 3; ++j) {
        float acc = fmul(cam.R[j], cam.T[0]);
        acc = ffma(cam.R[3 + j], cam.T[1], acc);
        acc = ffma(cam.R[6 + j], cam.T[2], acc);
        c[j] = -acc;
    }
}

// The camera centre -R^T T as hi + lo pairs (compensated, for view directions of km-scale scenes):
// a direction m - c is then (m - hi) - lo, exact to a few units in the last place of |m - c|.
__device__ __forceinline__ void camera_centre_pair(const h3dgs_camera& cam, float hi[3], float lo[3]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float h, l;
        dot2_pair(cam.R[j], cam.R[3 + j], cam.R[6 + j], 0.0f, cam.T[0], cam.T[1], cam.T[2], h, l);
        hi[j] = -h;
        lo[j] = -l;
    }
}

// Interpolation weight of the parent (Eq. t_interp); 0 unless eps_n < tau <= eps_p < inf.
__device__ __forceinline__ float parent_weight(float tau, float en, float ep) {
    if (!(en < tau) || !(ep >= tau) || isinf(ep)) return 0.0f;
    const float t = fdiv(fsub(tau, en), fsub(ep, en));
    return fminf(fmaxf(t, 0.0f), 1.0f);
}

// Pixel of thread `tid` inside a TW x TH tile: each warp owns an 8 x 4 block of pixels, so a warp
// can skip every splat whose alpha-floor box misses its block.
template <int TW, int TH>
__device__ __forceinline__ void tile_pixel(int tid, int& lx, int& ly) {
    constexpr int WX = TW / 8;
    const int w = tid >> 5, l = tid & 31;
    lx = (w % WX) * 8 + (l & 7);
    ly = (w / WX) * 4 + (l >> 3);
}

// Two pixels per thread: warp w owns the 8x8 block (w % (TW/8), w / (TW/8)) of the tile, lane l the
// pixels (l % 8, l / 8) and (l % 8, l / 8 + 4) of it.
template <int TW, int TH>
__device__ __forceinline__ void tile_pixel2(int tid, int& lx, int& ly0) {
    constexpr int WX = TW / 8;
    const int w = tid >> 5, l = tid & 31;
    lx = (w % WX) * 8 + (l & 7);
    ly0 = (w / WX) * 8 + (l >> 3);
}

// Whether the splat can reach alpha_floor at a pixel centre of the rectangle [x0, x1] x [y0, y1]
// (pixel-centre coordinates): the box test, then the minimum of q = -p2 over the rectangle (the
// centre if inside, else the best point of the four edges) against rz.  block_reach: the block
// [x0, x0 + BW - 1] x [y0, y0 + BH - 1].
__device__ __forceinline__ bool rect_reach(const float4 a, float cc, const float4 d, float x0, float y0, float x1,
                                           float y1) {
    const float hx = d.x, hy = d.y;
    if (!(hx >= 0.0f)) return false;
    const float u = a.x, v = a.y;
    if (!(u + hx >= x0 && u - hx <= x1 && v + hy >= y0 && v - hy <= y1)) return false;
    if (u >= x0 && u <= x1 && v >= y0 && v <= y1) return true;
    const float qa = -a.z, qb = -a.w, qc = -cc, rz = d.z;
    // edge minimisers use approximate reciprocals: a slightly moved point on the edge changes q only
    // to second order, far inside the 2% margin of rz
    const float kx = -qb * __fdividef(0.5f, qc), ky = -qb * __fdividef(0.5f, qa);
    const float dx0 = x0 - u, dx1 = x1 - u, dy0 = y0 - v, dy1 = y1 - v;
    float qmin = __int_as_float(0x7f800000);
#pragma unroll
    for (int e = 0; e < 2; ++e) {   // vertical edges: best dy = clamp(-qb dx / (2 qc))
        const float dx = e ? dx1 : dx0;
        const float dy = fminf(fmaxf(kx * dx, dy0), dy1);
        qmin = fminf(qmin, qa * dx * dx + qb * dx * dy + qc * dy * dy);
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {   // horizontal edges: best dx = clamp(-qb dy / (2 qa))
        const float dy = e ? dy1 : dy0;
        const float dx = fminf(fmaxf(ky * dy, dx0), dx1);
        qmin = fminf(qmin, qa * dx * dx + qb * dx * dy + qc * dy * dy);
    }
    return !(qmin > rz);   // NaN keeps the block
}
template <int BW, int BH>
__device__ __forceinline__ bool block_reach(const float4 a, float cc, const float4 d, float x0, float y0) {
    return rect_reach(a, cc, d, x0, y0, x0 + (float)(BW - 1), y0 + (float)(BH - 1));
}

// Bit w set if the splat can reach alpha_floor at a pixel centre of warp w's 8 x BH block in the tile
// with pixel origin (ox, oy); a clear bit means alpha < alpha_floor at every pixel of the block, so
// the warp would skip the splat anyway.  a = {u, v, ca, cb}, cc = the third conic term (pre-scaled:
// the exponent is p2 = ca dx^2 + cb dx dy + cc dy^2), d = {hx, hy, rz, z}: hx, hy are the inflated
// half-widths of the bounding box of the level set o_max 2^p2 = alpha_floor and rz = log2(o_max /
// alpha_floor) inflated by 2% + 0.02; hx < 0 marks a splat that never reaches the floor.
template <int TW, int TH, int BH = 4>
__device__ __forceinline__ uint32_t warp_mask(const float4 a, float cc, const float4 d, int ox, int oy) {
    constexpr int NW = TW * TH / (8 * BH), WX = TW / 8;
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w)
        if (block_reach<8, BH>(a, cc, d, (float)(ox + (w % WX) * 8) + 0.5f, (float)(oy + (w / WX) * BH) + 0.5f))
            m |= 1u << w;
    return m;
}

// The automatic blend chunk.  Splitting long lists into chunks shortens the critical path of a frame
// whose long lists are few among many short ones (a street view: lists of thousands of entries near
// the vanishing point, a mean of 94 to 165 per tile), but costs the producer/consumer hand-over, the
// scratch and a tail of consumers at the end of the queue, which is all loss when nearly every list
// is long (the 100M-node city at 1080p: a mean of 1115).  Measured with the split threshold at
// gamma x (pairs per resident CTA): the corridor is fastest when every list above 320 is split (1080p
// 0.454 ms, 4K 0.745 ms; 0.497 / 0.842 ms with gamma = 2), the city without any split (render
// 1.81 ms; 2.41 ms split at 320).  The rule: split at BLEND_AUTO_CHUNK while the frame's mean list
// length is at most BLEND_AUTO_MEAN_MAX, do not split above it.
constexpr int BLEND_AUTO_CHUNK = 320;
constexpr int BLEND_AUTO_MEAN_MAX = 450;
constexpr int BLEND_NO_SPLIT = 0x7fffffff;
__host__ __device__ inline int blend_auto_split(uint32_t n_pairs, int64_t n_tiles) {
    return (int64_t)n_pairs <= (int64_t)BLEND_AUTO_MEAN_MAX * n_tiles ? BLEND_AUTO_CHUNK : BLEND_NO_SPLIT;
}

// First list entry of chunk c when a tile's list [r.x, r.y) is split into nch chunks of near-equal
// length (lengths differ by at most one; chunk nch ends at r.y).
__device__ __forceinline__ int chunk_begin(int2 r, int nch, int c) {
    return r.x + (int)(((int64_t)(r.y - r.x) * c) / nch);
}

// Programmatic dependent launch: a kernel launched with launch_dependent() may start while the
// previous kernel of the stream is still running.  Such a kernel calls griddep_wait() (in every
// block, before any early exit) before it reads anything an earlier kernel wrote or writes anything
// an earlier kernel reads; griddep_launch_dependents() lets the next kernel start early.  Both are
// no-ops for a kernel launched normally.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Hardware approximations (PTX .approx instructions) used by the blend and its adjoint; both take
// every per-pixel decision through these same definitions.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// alpha' = 1 - (1 - ap)^(1/K) of a K-child transition given the clamped parent alpha ap (Eq. alphap);
// K = 2 in the cancellation-free form ap / (1 + sqrt(1 - ap)).  ap <= alpha_clamp < 1.
__device__ __forceinline__ float alpha_prime(float ap, float K) {
    if (K == 2.0f) return ap * rcp_approx(1.0f + sqrt_approx(1.0f - ap));
    return 1.0f - ex2_approx(__fdividef(lg2_approx(1.0f - ap), K));
}

// Bounded wait of one thread until *p >= want (acquire): at most `limit` polls, sleeping between
// polls after the first few.  Giving up sets FLAG_WAIT_TIMEOUT in *flags and returns false; the
// caller then goes on with what it has (its result is invalid and flagged), so no wait can hang.
__device__ __forceinline__ bool wait_geq(const uint32_t* p, uint32_t want, int limit, uint32_t* flags) {
    uint32_t v;
    int spins = 0;
    do {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        if (v >= want) return true;
        if (++spins > 32) __nanosleep(128);
    } while (spins < limit);
    atomicOr(flags, FLAG_WAIT_TIMEOUT);
    return false;
}

// Camera set-up of camera i of a batch: copies the raw camera and derives, in a fixed fp32 order,
//   c_j = -(R_0j T_0 + R_1j T_1 + R_2j T_2)  as -fmaf(R_2j, T_2, fmaf(R_1j, T_1, R_0j * T_0)),
//   f = max(fx, fy),  limx = (0.65 W) / fx,  limy = (0.65 H) / fy.
__device__ __forceinline__ void setup_camera(const CamBatch& b, int i, DevCam* __restrict__ out) {
    const h3dgs_camera& c = b.cam[i];
    DevCam d;
    for (int k = 0; k < 9; ++k) d.R[k] = c.R[k];
    for (int k = 0; k < 3; ++k) d.T[k] = c.T[k];
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
    d.width = c.width; d.height = c.height; d.znear = c.znear; d.tau = c.tau;
    camera_centre(c, d.c);
    camera_centre_pair(c, d.ch, d.cl);
    d.f = fmaxf(c.fx, c.fy);
    d.limx = fdiv(fmul(0.65f, (float)c.width), c.fx);
    d.limy = fdiv(fmul(0.65f, (float)c.height), c.fy);
    d.tiles_x = b.tiles_x[i];
    d.tiles_y = b.tiles_y[i];
    d.tile_base = b.tile_base[i];
    d.pix_base = b.pix_base[i];
    out[b.first + i] = d;
}

// Camera index of global entry m given the per-camera offsets (binary search, n_cams small).
__device__ __forceinline__ int find_cam(const int64_t* __restrict__ offs, int n_cams, int64_t m) {
    int lo = 0, hi = n_cams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(offs + mid) <= m) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- launchers (host side)
// cut.cu
cudaError_t launch_pack_records(const h3dgs_hierarchy& h, float4* rec, cudaStream_t s);
// Per row of 256 nodes of the one-camera scan: the parents' union box and largest side (see cut.cu).
int64_t cut_row_count(int64_t n);
cudaError_t launch_cut_row_bounds(const float4* rec, int64_t n, float4* rb, cudaStream_t s);
cudaError_t launch_camera_setup(const CamBatch& b, const DevOpts* opts, DevCam* cams, cudaStream_t s);
struct CutWork {
    uint32_t* mask;          // [n_cams][words]
    uint32_t* block_counts;  // [n_cams][G]
    int64_t* cam_totals;     // [n_cams + 1] raw (untruncated) exclusive offsets
    int blocks;              // G
    int64_t chunk;           // nodes per block
    int64_t words;           // mask words per camera
    uint32_t* lb_work;       // single-camera pass: look-back workspace (NULL: use the three-pass path)
    int64_t lb_words;
    h3dgs_camera cam0;       // single-camera pass: the raw camera (its derived values are computed in the kernel)
    int num_sms = 148;
    uint32_t* skipped_nodes = nullptr;   // single-camera pass: nodes of the rows skipped by the bound test
};
// Look-back words the single-camera cut needs for n nodes.
size_t cut_single_work_words(int64_t n);

// Traversal cut of one camera (large trees): visits only the cut and its ancestors.
constexpr int TR_MAX_LEVELS = 1024;   // descent steps (two levels each; deeper trees: FLAG_CUT_TRUNCATED)
// level table words: frontier sizes [TR_MAX_LEVELS + 1], the nodes visited inside blocks, 2 barrier words
constexpr int TR_LEVEL_WORDS = TR_MAX_LEVELS + 1 + 1 + 2;
struct TravArgs {
    const float4* rec;           // packed cut records [n][2]
    const int32_t* child_start;  // [n]
    int64_t n;
    uint32_t* front[2];          // frontier node ids, double-buffered [cap]
    float* feps[2];              // the parent's granularity of every frontier entry [cap]
    int64_t cap;                 // frontier capacity (n suffices for any tree)
    uint32_t* level_count;       // [TR_LEVEL_WORDS] frontier sizes per step, ...; zeroed per launch
    uint32_t* inner;             // = level_count + TR_MAX_LEVELS + 1: nodes visited from shared memory
    uint32_t* bar;               // = level_count + TR_MAX_LEVELS + 2: the grid barrier's 2 words
    uint32_t* mark;              // [(n + 31) / 32] cut bits: zero before, cleared again by the compaction
    float* tnode;                // [n] the parent weight of every cut node
    uint32_t* flags;
};
size_t cut_traverse_work_words(int64_t n);
int cut_traverse_grid(int num_sms);   // resident blocks of the cooperative descent (0: unavailable)
cudaError_t launch_cut_traverse(const TravArgs& a, const h3dgs_camera& cam, int grid, uint32_t* lb_work,
                                int64_t lb_words, int32_t* cut_ids, float* cut_t, int64_t* cut_offsets,
                                int64_t* cam_totals, int64_t capacity, cudaStream_t s);
cudaError_t launch_cut(const DevHier& h, const DevCam* cams, int n_cams, const CutWork& w, int32_t* cut_ids,
                       float* cut_t, int64_t* cut_offsets, int64_t capacity, uint32_t* flags, cudaStream_t s);

// preprocess.cu
constexpr int SPLAT_F4 = 4;      // float4 per splat record
struct SplatBufs {
    float4* rec;           // [cap][4]: {u, v, ca, cb}, {cc, on', op', t}, {r, g, b, K}, {hx, hy, rz, z} (z = view depth)
    uint2* rect;           // [cap]: (x0 | x1 << 16, y0 | y1 << 16)
    uint32_t* depth_key;   // [cap] fp32 depth bits, 0xffffffff when culled
    uint32_t* depth_hist;  // [4][256] digit histograms of the visible splats' depth keys (zeroed by the caller)
    uint32_t* tiles;       // [cap] tiles touched (0 when culled)
    uint32_t* n_splats;    // [1] min(M_total, cap)
    uint32_t* n_visible;   // [1]
};
cudaError_t launch_preprocess(const DevHier& h, const DevCam* cams, int n_cams, const DevOpts& o,
                              const int32_t* cut_ids, const float* cut_t, const int64_t* cut_offsets,
                              int64_t cap, const SplatBufs& sb, uint32_t* flags, int grid, cudaStream_t s);
cudaError_t launch_interpolate_export(const DevHier& h, int n_cams, const int32_t* cut_ids, const float* cut_t,
                                      const int64_t* cut_offsets, int interpolate, float* out, int64_t m_total,
                                      cudaStream_t s);

// sort.cu
constexpr size_t RADIX_HEADER_WORDS = 2048;   // tickets, kept count, pass histograms
struct SortWork {
    uint32_t* work;         // radix_work_words(n_cap) words: header, then look-back words per pass and tile
    size_t words;
    int num_sms;
    uint32_t* flags;        // device flag word (FLAG_WAIT_TIMEOUT)
};
size_t radix_work_words(int64_t n_cap);
// Stable LSD radix sort of n = *n_dev <= n_cap key/value pairs on key bits [0, bits).  The first pass
// reads (kin, vin) (vin NULL: values are the input positions), later passes alternate between (ka, va)
// and (kb, vb); *result_in_a tells which pair holds the result (kin/vin may alias kb/vb).  With
// drop_max, keys equal to 0xffffffff are left out; *n_kept (device) receives the number sorted.
// hist_pre: the digit histograms of every pass ([passes][256], 8-bit digits from the low end) already
// counted by the producer of the keys, with *n_kept already holding the number of kept keys; NULL:
// the sort counts them itself.
// pre_zeroed: the workspace (radix_work_words(n_cap) words) was cleared by the caller.
// ranges ([n_ranges][2], zeroed by the caller; NULL: not wanted): for every key value k < n_ranges
// present, {~first, last + 1} of its positions in the sorted output (the first position bit-inverted,
// so that an absent key stays {0, 0}; decode with ~).
cudaError_t radix_sort_pairs(const uint32_t* kin, const uint32_t* vin, uint32_t* ka, uint32_t* va, uint32_t* kb,
                             uint32_t* vb, const uint32_t* n_dev, int64_t n_cap, int bits, bool drop_max,
                             uint32_t* n_kept, const SortWork& w, bool* result_in_a, cudaStream_t s,
                             const uint32_t* hist_pre = nullptr, bool pre_zeroed = false, uint32_t* ranges = nullptr,
                             int64_t n_ranges = 0);
// Zeroes up to 8 regions of 32-bit words in one launch (the per-frame clears of the render).
struct ResetList {
    int n = 0;
    uint32_t* p[8];
    uint64_t words[8];
    DevCam* cams = nullptr;   // non-NULL: the launch also sets up the cameras of `cb` (one batch)
    CamBatch cb;
};
cudaError_t launch_reset(const ResetList& r, int num_sms, cudaStream_t s);
size_t pair_offsets_work_words(int64_t n_cap);
// Pair offsets of the depth order: pair_off[i] = sum of tiles[order[j]] over j < i (i < *n_dev <= n_cap),
// *total = the sum; seg_start[s] = the entry holding pair s DUP_SEG (for s < seg_cap).
constexpr int DUP_SEG = 1024;         // pairs per duplication block
cudaError_t launch_pair_offsets(const uint32_t* tiles, const uint32_t* order, const uint32_t* n_dev, int64_t n_cap,
                                uint32_t* pair_off, uint32_t* seg_start, int64_t seg_cap, uint32_t* total,
                                const SortWork& w, cudaStream_t s, bool pre_zeroed = false);
cudaError_t launch_pair_segments(const uint32_t* tiles, const uint32_t* order, const uint32_t* n_dev,
                                 const uint32_t* pair_off, uint32_t* seg_start, int64_t seg_cap, int grid,
                                 cudaStream_t s);
// Pairs (tile id, cut position) of the depth-ordered splats; *n_pairs_kept = min(*n_pairs, cap_pairs).
// hist (nullable, zeroed by the caller): the tile keys' digit histograms for hist_passes (<= 4) passes.
cudaError_t launch_duplicate(const DevCam* cams, int n_cams, const int64_t* cut_offsets, const SplatBufs& sb,
                             const uint32_t* order, const uint32_t* n_order, const uint32_t* pair_off,
                             const uint32_t* seg_start, const uint32_t* n_pairs, int64_t cap_pairs,
                             uint32_t* n_pairs_kept, uint32_t* keys, uint32_t* vals, uint32_t* hist, int hist_passes,
                             uint32_t* flags, cudaStream_t s);

// blend.cu
// Everything the chunked blend and its adjoint share.  Items are (tile, chunk) pairs; tiles with at
// most `chunk` list entries are one item.  Scratch holds, per (item, pixel), the chunk's (1 - alpha)
// product, colour, end transmittance and last contributor (split tiles only).
struct BlendArgs {
    const DevCam* cams;
    int n_cams;
    int64_t n_tiles;
    DevOpts o;
    int2* ranges;                 // as the tile sort leaves them ({~first, last + 1}); the plan decodes them
    const uint32_t* list;
    uint32_t* q_prod;             // blend queue: producer items (chunks 0 .. nch - 2 of split tiles)
    uint32_t* q_single;           // blend queue: single-chunk tiles
    uint32_t* q_cons;             // blend queue: consumer items (chunks 1 .. nch - 1 of split tiles)
    uint32_t* queue_sync;         // [1 + 2 n_tiles]: queue ticket, per-tile finished-producer counters, per-tile
                                  // finished middle-consumer counters
    const float4* splat;
    const uint32_t* n_splats;     // device: splat records written by the preprocess (bounds checks only)
    int chunk;                    // list entries per item, or 0: automatic (see blend_auto_chunk)
    const uint32_t* n_pairs;      // device: the frame's pairs (the automatic chunk)
    int64_t item_cap;
    int2* items;
    int32_t* tile_item0;
    int32_t* tile_nch;
    uint32_t* n_items;            // [4]: items, producers X, singles Y, split tiles
    float* scratch_Tc;
    float* scratch_C;
    float* scratch_Tend;
    int32_t* scratch_last;
    float* images;
    float* depth;                 // expected depth per pixel, or NULL (not computed)
    const float* exposure;        // [n_cams][12] row-major 3x4 exposure affines, or NULL (identity)
    float* scratch_D;             // per (item, pixel) expected depth of split tiles' chunks (depth only)
    float* T_final;
    int32_t* n_contrib;
    unsigned long long* n_evals;  // [5]: main-pass evaluations, middle producers' evaluations, main-pass
                                  // evaluations of splats with t != 0, applied contributions, those of
                                  // splats with t != 0
    uint32_t* work;               // look-back workspace of the plan (LB_HEADER_WORDS + 2 per 1024 tiles)
    size_t work_words;
    uint32_t* flags;              // device flag word
    cudaEvent_t* ev_queue;        // 2 events around the main blend kernel (profiling), or NULL
    bool pre_zeroed;              // work (the plan's look-back words) and queue_sync already cleared
    int num_sms;
};
size_t blend_plan_work_words(int64_t n_tiles);
cudaError_t launch_blend(const BlendArgs& a, cudaStream_t s);
// Test hook: one thread waits with wait_geq on *word (which nothing sets) for `polls` polls.
cudaError_t launch_wait_probe(const uint32_t* word, int polls, uint32_t* flags, cudaStream_t s);

// builder.cu
struct BuildOut {
    float *mean, *scale, *rot, *opacity, *sh, *box_min, *box_max;
    int32_t *parent, *child_start, *child_count;
};
// Options of one build: explicit leaf boxes ([L][6] min xyz, max xyz; NULL: the 3-sigma boxes of the
// leaf Gaussians), whether leaves take part in orientation matching, and an optional output of the
// node id of every leaf ([L]).
struct BuildExtra {
    const float* leaf_box = nullptr;
    bool orient_leaves = true;
    int32_t* leaf_node = nullptr;
};
// Builds the 2L - 1 node hierarchy over L leaves (synchronous on stream s).
cudaError_t build_hierarchy(int64_t L, const float* mean, const float* scale, const float* rot, const float* opacity,
                            const float* sh, const BuildOut& out, const SortWork& sw, int num_sms, cudaStream_t s,
                            const BuildExtra& ex = BuildExtra());
// Consolidated hierarchy of K chunks (leaves of chunk c: [off[c], off[c + 1]), host offsets):
// nodes [0, 2K - 1) are the top tree over the chunk roots (breadth-first; its leaves are the chunk
// roots), followed by every chunk's own hierarchy without its root, chunk after chunk.
cudaError_t build_hierarchy_chunked(int K, const int64_t* off, const float* mean, const float* scale, const float* rot,
                                    const float* opacity, const float* sh, const BuildOut& out, const SortWork& sw,
                                    int num_sms, cudaStream_t s);

// compact.cu
// Compaction of the resident hierarchy (h, rec) over the training cameras cams_host (host array).
// Writes *n_out = the number of kept nodes; when it exceeds `capacity` nothing else is written.
// Synchronous on stream s; allocates temporary device memory.
cudaError_t compact_hierarchy(const h3dgs_hierarchy& h, const float4* rec, const h3dgs_camera* cams_host,
                              int n_cams, const float* levels, int n_levels, const BuildOut& out, int64_t capacity,
                              int32_t* old_index, int64_t* n_out, const SortWork& sw, int num_sms, cudaStream_t s);

// stream.cu -- streamed hierarchy: attributes in page-locked host memory, a device cache of rows
struct StreamState {
    int64_t n_nodes, cap;                                     // nodes; cache rows
    const float *h_mean, *h_scale, *h_rot, *h_opacity, *h_sh;  // device mappings of the host arrays
    float *mean, *scale, *rot, *opacity, *sh;                  // cache rows [cap] (hierarchy layouts)
    int32_t* slot_of;    // [n_nodes] cache row, -1 absent (-2 while claimed by an update)
    int32_t* node_of;    // [cap] node of the row, -1 free
    int32_t* stamp;      // [cap] frame of the last update that needed the row
    int32_t* free_list;  // [cap] stack of free rows
    int32_t* missing;    // [n_nodes] nodes to transfer in the current update
    uint32_t* count;     // [4] free rows, listed nodes, transferred by the last update, requested by it
};
cudaError_t stream_init(const StreamState& st, int num_sms, cudaStream_t s);
cudaError_t stream_update(const StreamState& st, const int32_t* parent, int n_cams, const int32_t* cut_ids,
                          const float* cut_t, const int64_t* cut_offsets, int32_t frame, uint32_t* flags, int num_sms,
                          cudaStream_t s);
cudaError_t stream_cleanup(const StreamState& st, int32_t frame, int32_t max_age, int num_sms, cudaStream_t s);

// calib.cu: FP32 (paired FFMA) and exp2 (MUFU) rates of the running GPU, from chain kernels
cudaError_t measure_peaks(int num_sms, float* fp32_tflops, float* ex2_gops, cudaStream_t s);

// backward.cu
struct GradBufs {
    float* mean; float* scale; float* rot; float* opacity; float* sh;
};
cudaError_t launch_backward(const DevHier& h, const BlendArgs& a, const int32_t* cut_ids, const float* cut_t,
                            const int64_t* cut_offsets, const uint2* rect, const uint32_t* n_splats, const float* dL,
                            const float* dLdepth /* NULL: no depth gradient */, float* splat_grad, const GradBufs& g,
                            int freeze_leaves, int grid, cudaEvent_t* ev /* 4 events or NULL */, cudaStream_t s);

}  // namespace h3dgs
