// Per-tile front-to-back blending (a7).
//
// One CTA per screen tile, one thread per pixel.  The tile's splat list is consumed in batches
// staged through shared memory (one 48-byte record per thread per batch); every pixel walks the
// batch in order:
//   G = 2^(ca dx^2 + cb dx dy + cc dy^2)                (conic pre-scaled by -log2(e)/2)
//   alpha_n = min(c, o_n G),  alpha_p = min(c, o_p G)
//   alpha'  = 1 - (1 - alpha_p)^(1/K)                   (Eq. alphap; K = 2: alpha_p / (1 + sqrt(1 - alpha_p)))
//   alpha   = (1 - t) alpha_n + t alpha'                (t = parent weight; t = 0 skips alpha')
//   skip alpha < alpha_floor; stop before T (1 - alpha) < t_min; C += colour alpha T.
// The per-pixel decision quantities (dx, dy, exponent, alpha, T) use a fixed fp32 order; the
// exponential and alpha' use the fast hardware approximations.
#include "internal.cuh"

namespace h3dgs {

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

// alpha' of a K-child transition given the clamped parent alpha
__device__ __forceinline__ float alpha_prime(float ap, float K) {
    if (K == 2.0f) return __fdividef(ap, 1.0f + sqrtf(1.0f - ap));
    return 1.0f - ex2_approx(__fdividef(lg2_approx(1.0f - ap), K));
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) blend_kernel(const DevCam* __restrict__ cams, int n_cams, DevOpts o,
                                                        const int2* __restrict__ ranges, const uint32_t* __restrict__ list,
                                                        const float4* __restrict__ splat, float* __restrict__ images,
                                                        float* __restrict__ T_final, int32_t* __restrict__ n_contrib,
                                                        unsigned long long* __restrict__ n_evals) {
    constexpr int NT = TW * TH;
    __shared__ float4 s_a[NT], s_b[NT], s_c[NT];
    __shared__ unsigned int s_evals;
    const int64_t tile = blockIdx.x;
    if (threadIdx.x == 0) s_evals = 0;
    // camera of this tile
    int lo = 0, hi = n_cams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cams[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    const DevCam& cam = cams[lo];
    const int local = (int)(tile - cam.tile_base);
    const int tx = local % cam.tiles_x, ty = local / cam.tiles_x;
    const int px_i = tx * TW + (threadIdx.x % TW), py_i = ty * TH + (threadIdx.x / TW);
    const bool inside = px_i < cam.width && py_i < cam.height;
    const float px = (float)px_i + 0.5f, py = (float)py_i + 0.5f;
    const int2 r = ranges[tile];
    const float clampv = o.alpha_clamp, afloor = o.alpha_floor, tmin = o.t_min;
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    int last = 0;
    unsigned int evals = 0;
    bool done = !inside;
    for (int b0 = r.x; b0 < r.y; b0 += NT) {
        if (__syncthreads_count(done) == NT) break;
        const int n = min(NT, r.y - b0);
        if ((int)threadIdx.x < n) {
            const uint32_t s = __ldg(list + b0 + threadIdx.x);
            s_a[threadIdx.x] = __ldg(splat + 3 * (int64_t)s);
            s_b[threadIdx.x] = __ldg(splat + 3 * (int64_t)s + 1);
            s_c[threadIdx.x] = __ldg(splat + 3 * (int64_t)s + 2);
        }
        __syncthreads();
        if (!done) {
            for (int j = 0; j < n; ++j) {
                ++evals;
                const float4 a = s_a[j], b = s_b[j];
                const float dx = fsub(px, a.x), dy = fsub(py, a.y);
                const float h = ffma(a.z, dx, fmul(a.w, dy));
                const float g = fmul(fmul(b.x, dy), dy);
                const float p2 = ffma(dx, h, g);
                const float G = ex2_approx(p2);
                const float an = fminf(clampv, fmul(b.y, G));
                float alpha = an;
                if (b.w != 0.0f) {
                    const float ap = fminf(clampv, fmul(b.z, G));
                    const float apr = alpha_prime(ap, s_c[j].w);
                    alpha = ffma(b.w, apr, fmul(fsub(1.0f, b.w), an));
                }
                if (alpha < afloor) continue;
                const float Tn = fmul(T, fsub(1.0f, alpha));
                if (Tn < tmin) { done = true; break; }
                const float w = alpha * T;
                const float4 c = s_c[j];
                C0 = fmaf(c.x, w, C0);
                C1 = fmaf(c.y, w, C1);
                C2 = fmaf(c.z, w, C2);
                T = Tn;
                last = b0 + j + 1 - r.x;
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) evals += __shfl_down_sync(0xffffffffu, evals, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_evals, evals);
    __syncthreads();
    if (threadIdx.x == 0 && n_evals) atomicAdd(n_evals, (unsigned long long)s_evals);
    if (inside) {
        const int64_t pix = cam.pix_base + (int64_t)py_i * cam.width + px_i;
        const int64_t plane = (int64_t)cam.width * cam.height;
        float* img = images + 3 * cam.pix_base + (int64_t)py_i * cam.width + px_i;
        img[0] = fmaf(T, o.bg[0], C0);
        img[plane] = fmaf(T, o.bg[1], C1);
        img[2 * plane] = fmaf(T, o.bg[2], C2);
        if (T_final) T_final[pix] = T;
        if (n_contrib) n_contrib[pix] = last;
    }
}

cudaError_t launch_blend(const DevCam* cams, int n_cams, int64_t n_tiles, const DevOpts& o, const int2* ranges,
                         const uint32_t* list, const float4* splat, float* images, float* T_final, int32_t* n_contrib,
                         unsigned long long* n_evals, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)n_tiles;
    if (o.tile_w == 16 && o.tile_h == 16)
        blend_kernel<16, 16><<<grid, 256, 0, s>>>(cams, n_cams, o, ranges, list, splat, images, T_final, n_contrib, n_evals);
    else if (o.tile_w == 8 && o.tile_h == 8)
        blend_kernel<8, 8><<<grid, 64, 0, s>>>(cams, n_cams, o, ranges, list, splat, images, T_final, n_contrib, n_evals);
    else if (o.tile_w == 32 && o.tile_h == 8)
        blend_kernel<32, 8><<<grid, 256, 0, s>>>(cams, n_cams, o, ranges, list, splat, images, T_final, n_contrib, n_evals);
    else if (o.tile_w == 8 && o.tile_h == 32)
        blend_kernel<8, 32><<<grid, 256, 0, s>>>(cams, n_cams, o, ranges, list, splat, images, T_final, n_contrib, n_evals);
    else if (o.tile_w == 16 && o.tile_h == 8)
        blend_kernel<16, 8><<<grid, 128, 0, s>>>(cams, n_cams, o, ranges, list, splat, images, T_final, n_contrib, n_evals);
    else if (o.tile_w == 32 && o.tile_h == 4)
        blend_kernel<32, 4><<<grid, 128, 0, s>>>(cams, n_cams, o, ranges, list, splat, images, T_final, n_contrib, n_evals);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace h3dgs
