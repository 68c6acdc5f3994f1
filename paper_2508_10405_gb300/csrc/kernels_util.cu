// Small kernels around the time loop: model and perturbation preparation
// (Sec. 2 parameter map), residual injection, stacking of the per-shot images
// and the chain rule of Sec. 3, pseudo-Hessian stacking (App. B), the spike
// comb of App. D, the muted data residual of Sec. 4 and the FP64-accumulated
// vector kernels of the CGNR driver.
#include <algorithm>

#include "lsrtm_internal.cuh"

namespace lsrtm {
namespace {

constexpr int NT = 256;

__device__ __forceinline__ long long pad_of(const GridDev &g, long long k)
{
    long long ix = k % g.nx;
    long long t = k / g.nx;
    long long iy = t % g.ny;
    long long iz = t / g.ny;
    return (iz + g.z0) * g.rowz + (iy + g.y0) * (long long)g.pitch + (ix + g.x0);
}

__global__ void k_model_prep(GridDev g, const float *vp, const float *rho, float *kdt, float *binv)
{
    long long ncell = (long long)g.Nz * g.Ny * g.Nx;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        int x = (int)(c % g.Nx);
        long long t = c / g.Nx;
        int y = (int)(t % g.Ny);
        int z = (int)(t / g.Ny);
        // edge replication into the pad; above a free surface the mirror image
        int iz = z - g.z0;
        if (g.fs && iz < 0) iz = -iz;
        iz = min(max(iz, 0), g.nz - 1);
        int iy = min(max(y - g.y0, 0), g.ny - 1);
        int ix = min(max(x - g.x0, 0), g.nx - 1);
        long long k = ((long long)iz * g.ny + iy) * g.nx + ix;
        float v = vp[k], r = rho[k];
        long long p = (long long)z * g.rowz + (long long)y * g.pitch + x;
        kdt[p] = g.dt * r * v * v;
        binv[p] = 1.0f / r;
    }
}

// Perturbation map of Sec. 2 interleaved with the background coefficients:
// kd2 = (dt kappa, dt kappa (dlnVp + dlnIp)), br2 = (1/rho, (dlnIp - dlnVp)/rho),
// the perturbation parts zero outside the interior.
__global__ void k_pert_prep(GridDev g, const float *dm, const float *kdt, const float *binv,
                            float2 *kd2, float2 *br2)
{
    long long nint = (long long)g.nz * g.ny * g.nx;
    long long ncell = (long long)g.Nz * g.Ny * g.Nx;
    for (long long c0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; c0 < ncell;
         c0 += (long long)gridDim.x * blockDim.x) {
        int x = (int)(c0 % g.Nx);
        long long t = c0 / g.Nx;
        int y = (int)(t % g.Ny);
        int z = (int)(t / g.Ny);
        long long c = (long long)z * g.rowz + (long long)y * g.pitch + x;
        int iz = z - g.z0, iy = y - g.y0, ix = x - g.x0;
        // the perturbation lives on the interior; above a free surface its
        // mirror image, so ghost velocities are exact mirrors of live ones
        if (g.fs && iz < 0) iz = -iz;
        float dk = 0.f, dr = 0.f;
        if (iz >= 0 && iz < g.nz && iy >= 0 && iy < g.ny && ix >= 0 && ix < g.nx) {
            long long k = ((long long)iz * g.ny + iy) * g.nx + ix;
            float m1 = dm[k], m2 = dm[nint + k];
            dk = kdt[c] * (m1 + m2);
            dr = (m2 - m1) * binv[c];
        }
        kd2[c] = make_float2(kdt[c], dk);
        br2[c] = make_float2(binv[c], dr);
    }
}

__global__ void k_inject(GridDev g, TileRecs tr, int shot0, const float *dstage, int n, float2 *pl,
                         long long sstride2)
{
    int slot = blockIdx.y;
    int t = (shot0 + slot) * tr.ntiles + blockIdx.x;
    int b = tr.ptr[t], e = tr.ptr[t + 1];
    float2 *dst = pl + slot * sstride2;
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
        int2 rc = tr.rec[i];
        if (i > b && tr.rec[i - 1].x == rc.x) continue;
        float add = 0.f;
        for (int k = i; k < e && tr.rec[k].x == rc.x; ++k)
            add += dstage[(long long)tr.rec[k].y * g.nt + n];
        dst[rc.x].y += add;
    }
}

// Cell of interior point k (of the model grid gm) in slot b's grid g, or -1
// when it lies outside that shot's aperture window (win_x0 null: no windows,
// gm and g are the same grid).
__device__ inline long long slot_cell(const GridDev &gm, const GridDev &g, long long k, int shot,
                                      const int *win_x0, const int *win_nx)
{
    if (!win_x0) return pad_of(g, k);
    const int ix = (int)(k % gm.nx), iz = (int)(k / gm.nx);
    const int xl = ix - win_x0[shot];
    if (xl < 0 || xl >= win_nx[shot]) return -1;
    return (long long)(iz + g.z0) * g.pitch + g.x0 + xl;
}

__global__ void k_image_acc(GridDev gm, GridDev g, const float2 *img, int batch, int shot0, const int *win_x0,
                            const int *win_nx, double2 *acc)
{
    long long nint = (long long)gm.nz * gm.ny * gm.nx;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nint;
         k += (long long)gridDim.x * blockDim.x) {
        double2 s = acc[k];
        for (int b = 0; b < batch; ++b) {
            long long c = slot_cell(gm, g, k, shot0 + b, win_x0, win_nx);
            if (c < 0) continue;
            float2 v = img[b * g.plane + c];
            s.x += v.x;
            s.y += v.y;
        }
        acc[k] = s;
    }
}

// One CTA per (field, slot): scale = pow2_scale(max |band|) of the step's
// FP32 stage, then the scaled values in the 16-bit format.
__global__ void k_band_pack(Bands b, int shot0, int n)
{
    using lsrtm::pow2_scale;
    __shared__ float red[32];
    const int field = blockIdx.x, slot = blockIdx.y;
    const float *src = b.stage + ((long long)slot * 2 + field) * b.nb;
    float m = 0.f;
    for (long long i = threadIdx.x; i < b.nb; i += blockDim.x) m = fmaxf(m, fabsf(src[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) red[0] = m;
    }
    __syncthreads();
    const float sc = pow2_scale(red[0]);
    const float inv = 1.0f / sc;   // exact: a power of two
    const long long row = band_row(b, shot0 + slot, n);
    if (threadIdx.x == 0) b.scale[row * 2 + field] = sc;
    void *dst = field ? b.v : b.p;
    const long long o = row * b.nb;
    if (b.fmt == BAND_BF16S) {
        __nv_bfloat16 *d = reinterpret_cast<__nv_bfloat16 *>(dst) + o;
        for (long long i = threadIdx.x; i < b.nb; i += blockDim.x) d[i] = __float2bfloat16_rn(src[i] * inv);
    } else {
        __half *d = reinterpret_cast<__half *>(dst) + o;
        for (long long i = threadIdx.x; i < b.nb; i += blockDim.x) d[i] = __float2half_rn(src[i] * inv);
    }
}

// g_kappa = -dt kappa sum_n Q lp, g_rho = (dt / 2) / rho * sum_n (products at
// the adjacent half nodes); g_Vp = g_kappa - g_rho, g_Ip = g_kappa + g_rho.
__global__ void k_image_fin(GridDev g, const double2 *acc, const float *kdt, const float *binv,
                            float *gout)
{
    long long nint = (long long)g.nz * g.ny * g.nx;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nint;
         k += (long long)gridDim.x * blockDim.x) {
        long long c = pad_of(g, k);
        double gk = -(double)kdt[c] * acc[k].x;
        double gr = 0.5 * (double)g.dt * (double)binv[c] * acc[k].y;
        gout[k] = (float)(gk - gr);
        gout[nint + k] = (float)(gk + gr);
    }
}

__global__ void k_hess_acc(GridDev gm, GridDev g, const float *hess, int batch, int shot0, const int *win_x0,
                           const int *win_nx, double *acc)
{
    long long nint = (long long)gm.nz * gm.ny * gm.nx;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nint;
         k += (long long)gridDim.x * blockDim.x) {
        double s = acc[k];
        for (int b = 0; b < batch; ++b) {
            long long c = slot_cell(gm, g, k, shot0 + b, win_x0, win_nx);
            if (c >= 0) s += hess[b * g.plane + c];
        }
        acc[k] = s;
    }
}

__global__ void k_hess_fin(long long nint, const double *acc, float *out)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nint;
         k += (long long)gridDim.x * blockDim.x)
        out[k] = (float)acc[k];
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block-level FP64 sum of x*y (w optional), one partial per block.
__global__ void k_dot_partial(const float *x, const float *y, const float *w, long long n,
                              double *part)
{
    __shared__ double sh[NT / 32];
    double acc = 0.0;
    long long n4 = n / 4;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const float4 *y4 = reinterpret_cast<const float4 *>(y);
    const float4 *w4 = reinterpret_cast<const float4 *>(w);
    bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) |
                 reinterpret_cast<uintptr_t>(w)) & 15) == 0;
    long long start = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    if (vec) {
        for (long long i = start; i < n4; i += stride) {
            float4 a = x4[i], b = y4[i];
            if (w) {
                float4 c = w4[i];
                acc += (double)a.x * b.x * c.x + (double)a.y * b.y * c.y +
                       (double)a.z * b.z * c.z + (double)a.w * b.w * c.w;
            } else {
                acc += (double)a.x * b.x + (double)a.y * b.y + (double)a.z * b.z + (double)a.w * b.w;
            }
        }
        for (long long i = 4 * n4 + start; i < n; i += stride)
            acc += (double)x[i] * y[i] * (w ? (double)w[i] : 1.0);
    } else {
        for (long long i = start; i < n; i += stride)
            acc += (double)x[i] * y[i] * (w ? (double)w[i] : 1.0);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < NT / 32 ? sh[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

__global__ void k_sum_final(const double *part, int np, double *out)
{
    __shared__ double sh[NT / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < NT / 32 ? sh[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) *out = v;
    }
}

__global__ void k_maxabs(const float *x, long long n, float *out)
{
    __shared__ float sh[NT / 32];
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < NT / 32 ? sh[threadIdx.x] : 0.f;
        v = warp_max(v);
        // non-negative floats compare like their bit patterns as ints
        if (threadIdx.x == 0) atomicMax(reinterpret_cast<int *>(out), __float_as_int(v));
    }
}

__global__ void k_nonfinite(const float *x, long long n, int *flag)
{
    int bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    bad = __syncthreads_or(bad);
    if (bad && threadIdx.x == 0) atomicOr(flag, 1);
}

// Non-finite guard over the first count4 float4s of each slot (blockIdx.y):
// a float is NaN or Inf exactly when its eight exponent bits are all ones.
// A tripped word is left as it is (the first detection names the step).
__global__ void k_guard_state(const float4 *x, long long stride4, long long count4, int *word, int code)
{
    __shared__ int tripped;
    if (threadIdx.x == 0) tripped = *reinterpret_cast<volatile int *>(word);
    __syncthreads();
    if (tripped) return;
    const float4 *xs = x + blockIdx.y * stride4;
    unsigned bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count4;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 v = xs[i];
        const unsigned e = 0x7f800000u;
        bad |= ((__float_as_uint(v.x) & e) == e) | ((__float_as_uint(v.y) & e) == e) |
               ((__float_as_uint(v.z) & e) == e) | ((__float_as_uint(v.w) & e) == e);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(word, 0, code);
}

// 16-bit checkpoint planes. Plane q of slot s of a snapshot is stored as
// v / c with c = pow2_scale(m), m = max|plane|: m is taken first
// (k_ck_absmax; the bits of non-negative floats order like the floats),
// then k_ck_pack writes the scaled values and k_ck_unpack multiplies back.
// amax: [slot][ck_planes] of the snapshot.
__device__ __forceinline__ float ck_scale(float m) { return pow2_scale(m); }

__global__ void k_ck_absmax(const float *src, long long sstride, long long plane, float *amax, int ck_planes,
                            int p0)
{
    const float *x = src + blockIdx.z * sstride + blockIdx.y * plane;
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane;
         i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? wm[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0)
            atomicMax(reinterpret_cast<int *>(amax + blockIdx.z * ck_planes + p0 + blockIdx.y), __float_as_int(m));
    }
}

template <class H>
__device__ __forceinline__ H to16(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to16<__half>(float v) { return __float2half_rn(v); }
__device__ __forceinline__ float from16(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float from16(__half v) { return __half2float(v); }

template <class H>
__global__ void k_ck_pack(const float *src, long long sstride, long long plane, const float *amax, int ck_planes,
                          int p0, H *dst)
{
    const float *x = src + blockIdx.z * sstride + blockIdx.y * plane;
    const int q = p0 + blockIdx.y;
    H *o = dst + ((long long)blockIdx.z * ck_planes + q) * plane;
    const float inv = 1.f / ck_scale(amax[blockIdx.z * ck_planes + q]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane;
         i += (long long)gridDim.x * blockDim.x)
        o[i] = to16<H>(x[i] * inv);
}

template <class H>
__global__ void k_ck_unpack(float *dst, long long sstride, long long plane, const float *amax, int ck_planes, int p0,
                            const H *src)
{
    float *x = dst + blockIdx.z * sstride + blockIdx.y * plane;
    const int q = p0 + blockIdx.y;
    const H *i16 = src + ((long long)blockIdx.z * ck_planes + q) * plane;
    const float c = ck_scale(amax[blockIdx.z * ck_planes + q]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane;
         i += (long long)gridDim.x * blockDim.x)
        x[i] = c * from16(i16[i]);
}

__global__ void k_guard_scalars(const double *v, int n, int *word, int code)
{
    bool bad = false;
    for (int i = threadIdx.x; i < n; i += blockDim.x) bad |= !isfinite(v[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(word, 0, code);
}

// out[r][n] = mask(r, n) (dobs[r][n] - dsyn[r][n]). The direct-wave mute of
// receiver r is 0 before sample n0[r] (the first sample after the mute time,
// decided in FP64 on the host), then the raised-cosine rise
// (1 - cos(pi v)) / 2, v = (n - n0) b + a0[r] (the time past the mute time
// over the taper width), 1 from v >= 1 on (b = 0: a step); fo[r] is the
// far-offset factor. One block per receiver row at a time, threads along the
// samples, four samples per thread access when the rows are 16-byte aligned.
__device__ __forceinline__ float mute_factor(int n, int n0, float a0, float b, float f)
{
    if (n < n0) return 0.f;
    const float v = fmaf((float)(n - n0), b, a0);
    return (b <= 0.f || v >= 1.f) ? f : f * (0.5f * (1.f - cospif(v)));
}

template <bool VEC>
__global__ void k_mute_residual(const float *dobs, const float *dsyn, const int *n0, const float *a0,
                                const float *fo, long long nrec, int nt, float b, float *out)
{
    for (long long r = blockIdx.x; r < nrec; r += gridDim.x) {
        const int s0 = n0[r];
        const float a = a0[r], f = fo[r];
        const long long base = r * nt;
        if (VEC) {
            const float4 *o4 = reinterpret_cast<const float4 *>(dobs + base);
            const float4 *s4 = reinterpret_cast<const float4 *>(dsyn + base);
            float4 *w4 = reinterpret_cast<float4 *>(out + base);
            for (int q = threadIdx.x; q < nt / 4; q += blockDim.x) {
                float4 d = o4[q];
                if (dsyn) {
                    const float4 e = s4[q];
                    d.x -= e.x, d.y -= e.y, d.z -= e.z, d.w -= e.w;
                }
                const int n = 4 * q;
                d.x *= mute_factor(n, s0, a, b, f);
                d.y *= mute_factor(n + 1, s0, a, b, f);
                d.z *= mute_factor(n + 2, s0, a, b, f);
                d.w *= mute_factor(n + 3, s0, a, b, f);
                w4[q] = d;
            }
        } else {
            for (int n = threadIdx.x; n < nt; n += blockDim.x) {
                const float d = dsyn ? dobs[base + n] - dsyn[base + n] : dobs[base + n];
                out[base + n] = mute_factor(n, s0, a, b, f) * d;
            }
        }
    }
}

__global__ void k_comb(GridDev g, int param, int spacing, float *m)
{
    long long nint = (long long)g.nz * g.ny * g.nx;
    int h = spacing / 2;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nint;
         k += (long long)gridDim.x * blockDim.x) {
        int ix = (int)(k % g.nx);
        long long t = k / g.nx;
        int iy = (int)(t % g.ny);
        int iz = (int)(t / g.ny);
        bool on = (iz >= h && (iz - h) % spacing == 0) && (ix >= h && (ix - h) % spacing == 0) &&
                  (g.ndim == 2 || (iy >= h && (iy - h) % spacing == 0));
        m[k] = (param == 0 && on) ? 1.f : 0.f;
        m[nint + k] = (param == 1 && on) ? 1.f : 0.f;
    }
}

__global__ void k_axpy_ratio(float *x, const float *p, const double *num, const double *den,
                             float sign, long long n)
{
    double d = *den;
    float alpha = d != 0.0 ? (float)(*num / d) * sign : 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        x[i] += alpha * p[i];
}

__global__ void k_xpby_ratio(float *p, const float *z, const double *num, const double *den,
                             long long n)
{
    double d = *den;
    float beta = d != 0.0 ? (float)(*num / d) : 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

// x[plane][k] *= (mask bit of plane) * (w ? w[plane][k] : 1)
__global__ void k_mul_mask(float *x, const float *w, int mask, long long nint)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 2 * nint;
         i += (long long)gridDim.x * blockDim.x) {
        int plane = i >= nint;
        float f = ((mask >> plane) & 1) ? 1.f : 0.f;
        if (w) f *= w[i];
        x[i] *= f;
    }
}

__global__ void k_copy(float *dst, const float *src, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// minv = 1 / (h + eps * max(h)) for both planes
__global__ void k_precond(const float *h, const float *hmax, float eps, long long nint, float *minv)
{
    float hm = *hmax;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nint;
         i += (long long)gridDim.x * blockDim.x) {
        float v = 1.0f / (h[i] + eps * hm);
        minv[i] = v;
        minv[nint + i] = v;
    }
}

// rmap[rcell[q]] = q for the first entry q of every run of equal cells in [q0, q1).
__global__ void k_rmap_scatter(int *rmap, const int *rcell, int q0, int q1)
{
    for (int q = q0 + blockIdx.x * blockDim.x + threadIdx.x; q < q1; q += gridDim.x * blockDim.x)
        if (q == q0 || rcell[q - 1] != rcell[q]) rmap[rcell[q]] = q;
}

int grid_for(long long n)
{
    long long b = (n + NT - 1) / NT;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

}  // namespace

cudaError_t launch_model_prep(const GridDev &g, const float *vp, const float *rho, float *kdt,
                              float *binv, cudaStream_t s)
{
    long long n = (long long)g.Nz * g.Ny * g.Nx;
    k_model_prep<<<grid_for(n), NT, 0, s>>>(g, vp, rho, kdt, binv);
    return cudaGetLastError();
}

cudaError_t launch_pert_prep(const GridDev &g, const float *dm, const float *kdt,
                             const float *binv, float2 *kd2, float2 *br2, cudaStream_t s)
{
    long long n = (long long)g.Nz * g.Ny * g.Nx;
    k_pert_prep<<<grid_for(n), NT, 0, s>>>(g, dm, kdt, binv, kd2, br2);
    return cudaGetLastError();
}

cudaError_t launch_inject_residual(const GridDev &g, const TileRecs &tr, int batch, int shot0,
                                   const float *dstage, int n, float2 *pl, long long sstride2,
                                   cudaStream_t s)
{
    dim3 grid(tr.ntiles, batch);
    k_inject<<<grid, 64, 0, s>>>(g, tr, shot0, dstage, n, pl, sstride2);
    return cudaGetLastError();
}

cudaError_t launch_image_accumulate(const GridDev &gm, const GridDev &g, const float2 *img, int batch, int shot0,
                                    const int *win_x0, const int *win_nx, double2 *acc, cudaStream_t s)
{
    long long n = (long long)gm.nz * gm.ny * gm.nx;
    k_image_acc<<<grid_for(n), NT, 0, s>>>(gm, g, img, batch, shot0, win_x0, win_nx, acc);
    return cudaGetLastError();
}

cudaError_t launch_band_pack(const Bands &b, int batch, int shot0, int n, cudaStream_t s)
{
    k_band_pack<<<dim3(2, batch), 512, 0, s>>>(b, shot0, n);
    return cudaGetLastError();
}

cudaError_t launch_image_finalize(const GridDev &g, const double2 *acc, const float *kdt,
                                  const float *binv, float *gout, cudaStream_t s)
{
    long long n = (long long)g.nz * g.ny * g.nx;
    k_image_fin<<<grid_for(n), NT, 0, s>>>(g, acc, kdt, binv, gout);
    return cudaGetLastError();
}

cudaError_t launch_hess_accumulate(const GridDev &gm, const GridDev &g, const float *hess, int batch, int shot0,
                                   const int *win_x0, const int *win_nx, double *acc, cudaStream_t s)
{
    long long n = (long long)gm.nz * gm.ny * gm.nx;
    k_hess_acc<<<grid_for(n), NT, 0, s>>>(gm, g, hess, batch, shot0, win_x0, win_nx, acc);
    return cudaGetLastError();
}

cudaError_t launch_hess_finalize(const GridDev &g, const double *acc, float *out, cudaStream_t s)
{
    long long n = (long long)g.nz * g.ny * g.nx;
    k_hess_fin<<<grid_for(n), NT, 0, s>>>(n, acc, out);
    return cudaGetLastError();
}

cudaError_t launch_max_abs_reduce(const float *x, long long n, float *out, cudaStream_t s)
{
    k_maxabs<<<grid_for(n), NT, 0, s>>>(x, n, out);
    return cudaGetLastError();
}

cudaError_t launch_mute_residual(const float *dobs, const float *dsyn, const int *n0, const float *a0,
                                 const float *fo, long long nrec, int nt, float b, float *out, cudaStream_t s)
{
    if (nrec <= 0 || nt <= 0) return cudaSuccess;
    const int blocks = (int)std::min<long long>(nrec, 152 * 16);
    const bool vec = nt % 4 == 0 &&
                     ((reinterpret_cast<uintptr_t>(dobs) | reinterpret_cast<uintptr_t>(dsyn) |
                       reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    if (vec) k_mute_residual<true><<<blocks, NT, 0, s>>>(dobs, dsyn, n0, a0, fo, nrec, nt, b, out);
    else k_mute_residual<false><<<blocks, NT, 0, s>>>(dobs, dsyn, n0, a0, fo, nrec, nt, b, out);
    return cudaGetLastError();
}

cudaError_t launch_nonfinite_count(const float *x, long long n, int *flag, cudaStream_t s)
{
    k_nonfinite<<<grid_for(n), NT, 0, s>>>(x, n, flag);
    return cudaGetLastError();
}

cudaError_t launch_guard_state(const float *base, long long stride, long long count, int nslots, int *word,
                               int code, cudaStream_t s)
{
    if (nslots <= 0 || count <= 0) return cudaSuccess;
    const long long count4 = count / 4;
    // about four CTAs per SM over all slots
    const int gx = (int)std::max(1LL, std::min((count4 + NT - 1) / NT, (long long)std::max(1, 608 / nslots)));
    k_guard_state<<<dim3(gx, nslots), NT, 0, s>>>(reinterpret_cast<const float4 *>(base), stride / 4, count4, word,
                                                   code);
    return cudaGetLastError();
}

cudaError_t launch_ck_pack(const float *src, long long sstride, long long plane, int planes, int p0, int bs,
                           int ck_planes, int fmt, void *dst, float *amax, cudaStream_t s)
{
    if (bs <= 0 || planes <= 0) return cudaSuccess;
    const int gx = (int)std::max(1LL, std::min((plane + NT - 1) / NT, (long long)std::max(1, 608 / (planes * bs))));
    const dim3 grid(gx, planes, bs);
    // the maxima of these planes start from zero
    cudaError_t e = cudaMemset2DAsync(amax + p0, ck_planes * sizeof(float), 0, planes * sizeof(float), bs, s);
    if (e != cudaSuccess) return e;
    k_ck_absmax<<<grid, NT, 0, s>>>(src, sstride, plane, amax, ck_planes, p0);
    if (fmt == BAND_BF16S)
        k_ck_pack<<<grid, NT, 0, s>>>(src, sstride, plane, amax, ck_planes, p0, static_cast<__nv_bfloat16 *>(dst));
    else
        k_ck_pack<<<grid, NT, 0, s>>>(src, sstride, plane, amax, ck_planes, p0, static_cast<__half *>(dst));
    return cudaGetLastError();
}

cudaError_t launch_ck_unpack(float *dst, long long sstride, long long plane, int planes, int p0, int bs,
                             int ck_planes, int fmt, const void *src, const float *amax, cudaStream_t s)
{
    if (bs <= 0 || planes <= 0) return cudaSuccess;
    const int gx = (int)std::max(1LL, std::min((plane + NT - 1) / NT, (long long)std::max(1, 608 / (planes * bs))));
    const dim3 grid(gx, planes, bs);
    if (fmt == BAND_BF16S)
        k_ck_unpack<<<grid, NT, 0, s>>>(dst, sstride, plane, amax, ck_planes, p0,
                                        static_cast<const __nv_bfloat16 *>(src));
    else
        k_ck_unpack<<<grid, NT, 0, s>>>(dst, sstride, plane, amax, ck_planes, p0, static_cast<const __half *>(src));
    return cudaGetLastError();
}

cudaError_t launch_guard_scalars(const double *v, int n, int *word, int code, cudaStream_t s)
{
    k_guard_scalars<<<1, 32, 0, s>>>(v, n, word, code);
    return cudaGetLastError();
}

cudaError_t launch_rmap_scatter(int *rmap, const int *rcell, int q0, int q1, cudaStream_t s)
{
    if (q1 <= q0) return cudaSuccess;
    k_rmap_scatter<<<grid_for(q1 - q0), NT, 0, s>>>(rmap, rcell, q0, q1);
    return cudaGetLastError();
}

cudaError_t launch_comb(const GridDev &g, int param, int spacing, float *m, cudaStream_t s)
{
    long long n = (long long)g.nz * g.ny * g.nx;
    k_comb<<<grid_for(n), NT, 0, s>>>(g, param, spacing, m);
    return cudaGetLastError();
}

static constexpr int kDotBlocks = 152 * 4;

cudaError_t launch_dot(const float *x, const float *y, long long n, double *out, double *work,
                       cudaStream_t s)
{
    return launch_dot_w(x, y, nullptr, n, out, work, s);
}

cudaError_t launch_dot_w(const float *x, const float *y, const float *w, long long n,
                         double *out, double *work, cudaStream_t s)
{
    int nb = grid_for(n) < kDotBlocks ? grid_for(n) : kDotBlocks;
    k_dot_partial<<<nb, NT, 0, s>>>(x, y, w, n, work);
    k_sum_final<<<1, NT, 0, s>>>(work, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_axpy_ratio(float *x, const float *p, const double *num, const double *den,
                              float sign, long long n, cudaStream_t s)
{
    k_axpy_ratio<<<grid_for(n), NT, 0, s>>>(x, p, num, den, sign, n);
    return cudaGetLastError();
}

cudaError_t launch_xpby_ratio(float *p, const float *z, const double *num, const double *den,
                              long long n, cudaStream_t s)
{
    k_xpby_ratio<<<grid_for(n), NT, 0, s>>>(p, z, num, den, n);
    return cudaGetLastError();
}

cudaError_t launch_mul_mask(float *x, const float *w, int param_mask, long long nint,
                            cudaStream_t s)
{
    k_mul_mask<<<grid_for(2 * nint), NT, 0, s>>>(x, w, param_mask, nint);
    return cudaGetLastError();
}

cudaError_t launch_scale_copy(float *dst, const float *src, long long n, cudaStream_t s)
{
    k_copy<<<grid_for(n), NT, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

cudaError_t launch_precond_build(const float *h, const float *hmax, float eps, long long nint,
                                 float *minv, cudaStream_t s)
{
    k_precond<<<grid_for(nint), NT, 0, s>>>(h, hmax, eps, nint, minv);
    return cudaGetLastError();
}

}  // namespace lsrtm
