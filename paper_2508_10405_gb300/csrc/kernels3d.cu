// 3D time-step kernels for the staggered-grid Born operator and its exact
// transpose (Eq. 1, Eq. scattereqln, App. A).
//
// Each time step is two launches over all shots of a batch, one thread per
// padded cell, updating the state in place:
//   forward  k3_v (half nodes: v_x, v_y, v_z and their CPML memories from
//            D+ p) then k3_p (nodes: p from D- . v, source, records, bands);
//   adjoint  k3_a (half nodes: lambda_v, lambda_psi_p, background v^{n-1/2},
//            rho-image products at the half nodes) then k3_b (nodes:
//            lambda_p, lambda_psi_v, background p^{n-1}, residual injection
//            and the kappa image of step n-1).
// Stencil neighbours come through L1/L2. As in 2D, a background field and its
// partner (scattered or adjoint) are float2 pairs, so the stencils run as
// packed FFMA2. The adjoint fields are kept pre-scaled by the coefficient
// their neighbours' stencils apply: the node pair holds (p, mu) with
// mu = dt kappa lambda_p and the half-node pairs (v_d, w_d) with
// w_d = dt b_d lambda_v,d, so a stencil tap is one pair load; each stage
// recovers its own lambda with one division.
#include <algorithm>
#include <type_traits>

#include "lsrtm_internal.cuh"

namespace lsrtm {
namespace {

// Slot layouts in float planes (state updated in place).
// Born pairs (background, scattered): p vx vy vz | psi_p x y z | psi_v x y z.
enum { B3_P = 0, B3_V = 2, B3_PP = 8, B3_PV = 14 };   // B3_V + 2d, B3_PP + 2d, B3_PV + 2d
// Background only: p vx vy vz | psi_p x y z | psi_v x y z | (bu G)^2 x y z.
enum { G3_P = 0, G3_V = 1, G3_PP = 4, G3_PV = 7, G3_HQ = 10 };   // + d
// Adjoint pairs (background, lambda) p vx vy vz | lambda_psi_p x y z | lambda_psi_v x y z |
// kappa image (node) | rho image products at the half nodes x y z.
enum { A3_PL = 0, A3_V = 2, A3_LPP = 8, A3_LPV = 11, A3_IMK = 14, A3_IM = 15 };

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 fma_(float a, float2 b, float2 c) { return __ffma2_rn(f2(a), b, c); }
__device__ __forceinline__ float add_(float a, float b) { return a + b; }
__device__ __forceinline__ float2 add_(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float mul_(float a, float b) { return a * b; }
__device__ __forceinline__ float2 mul_(float a, float2 b) { return __fmul2_rn(f2(a), b); }
__device__ __forceinline__ float sub_(float a, float b) { return a - b; }
__device__ __forceinline__ float2 sub_(float2 a, float2 b) { return __ffma2_rn(f2(-1.f), b, a); }
template <class T> __device__ __forceinline__ T zero_();
template <> __device__ __forceinline__ float zero_<float>() { return 0.f; }
template <> __device__ __forceinline__ float2 zero_<float2>() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ float xof(float v) { return v; }
__device__ __forceinline__ float xof(float2 v) { return v.x; }
__device__ __forceinline__ float yof(float) { return 0.f; }
__device__ __forceinline__ float yof(float2 v) { return v.y; }

template <int M, class T, class F>
__device__ __forceinline__ T diff(const float *c, F f)   // sum_l c_l (f(l) - f(1 - l)) as (a_l, b_l) pairs
{
    T d[M];
#pragma unroll
    for (int l = 0; l < M; ++l) d[l] = f(l + 1);
    T acc = mul_(c[0], d[0]);
#pragma unroll
    for (int l = 1; l < M; ++l) acc = fma_(c[l], d[l], acc);
    return acc;
}

struct Cell {
    int x, y, z, slot;
    bool ok;
};

__device__ __forceinline__ Cell cell_of(const GridDev &g)
{
    Cell c;
    c.x = blockIdx.x * blockDim.x + threadIdx.x;
    c.y = blockIdx.y * blockDim.y + threadIdx.y;
    c.z = blockIdx.z % g.Nz;
    c.slot = blockIdx.z / g.Nz;
    c.ok = c.x < g.Nx && c.y < g.Ny;
    return c;
}

__device__ __forceinline__ int coord(const Cell &c, int d) { return d == 0 ? c.z : (d == 1 ? c.y : c.x); }
__device__ __forceinline__ int extent(const GridDev &g, int d) { return d == 0 ? g.Nz : (d == 1 ? g.Ny : g.Nx); }
__device__ __forceinline__ int origin(const GridDev &g, int d) { return d == 0 ? g.z0 : (d == 1 ? g.y0 : g.x0); }
__device__ __forceinline__ int inner(const GridDev &g, int d) { return d == 0 ? g.nz : (d == 1 ? g.ny : g.nx); }
__device__ __forceinline__ long long stride(const GridDev &g, int d)
{
    return d == 0 ? g.rowz : (d == 1 ? (long long)g.pitch : 1LL);
}
__device__ __forceinline__ const float *cdir(const GridDev &g, int d) { return d == 0 ? g.cz : (d == 1 ? g.cy : g.cx); }

// Face bands: [x faces 2M nz ny][y faces 2M nz nx][z faces 2M ny nx]; s in [0, 2M).
__device__ __forceinline__ long long face_index(const GridDev &g, int d, int iz, int iy, int ix, int s)
{
    const int M = g.M;
    if (d == 2) return ((long long)iz * g.ny + iy) * (2 * M) + s;
    long long base = 2LL * M * g.nz * g.ny;
    if (d == 1) return base + ((long long)iz * (2 * M) + s) * g.nx + ix;
    base += 2LL * M * g.nz * g.nx;
    return base + ((long long)s * g.ny + iy) * g.nx + ix;
}

// Band slot of the d-normal strip point (iz, iy, ix), -1 if not in the d face band.
__device__ __forceinline__ long long face_band(const GridDev &g, int d, int iz, int iy, int ix)
{
    const int M = g.M;
    int i = d == 0 ? iz : (d == 1 ? iy : ix);
    int n = inner(g, d);
    int s;
    if (i >= -M && i < 0) s = i + M;
    else if (i >= n && i < n + M) s = M + (i - n);
    else return -1;
    // the two other coordinates must be interior
    if (d != 0 && (iz < 0 || iz >= g.nz)) return -1;
    if (d != 1 && (iy < 0 || iy >= g.ny)) return -1;
    if (d != 2 && (ix < 0 || ix >= g.nx)) return -1;
    return face_index(g, d, iz, iy, ix, s);
}

__device__ __forceinline__ long long pband3(const GridDev &g, int iz, int iy, int ix)
{
    for (int d = 0; d < 3; ++d) {
        long long b = face_band(g, d, iz, iy, ix);
        if (b >= 0) return b;
    }
    return -1;
}


__device__ __forceinline__ bool pml_half(const GridDev &g, int d, int i)
{
    int o = origin(g, d);
    return (i <= o - 2) || (i >= o + inner(g, d));
}
__device__ __forceinline__ bool pml_node(const GridDev &g, int d, int i)
{
    int o = origin(g, d);
    return (i <= o - 1) || (i >= o + inner(g, d));
}

// ---------------------------------------------------------------------------
// Forward velocity stage (half nodes), in place.
// ---------------------------------------------------------------------------
template <int M, bool BORN, bool BANDS, bool HESS>
__global__ void __launch_bounds__(256) k3_v(const Step3D a)
{
    using T = typename std::conditional<BORN, float2, float>::type;
    using R = typename std::conditional<BORN, float2, float>::type;
    const GridDev &g = a.g;
    const Cell c = cell_of(g);
    if (!c.ok) return;
    const long long plane = g.plane;
    const long long cc = (long long)c.z * g.rowz + (long long)c.y * g.pitch + c.x;
    float *st = a.st + c.slot * a.sstride;
    T *S = reinterpret_cast<T *>(st);
    const T *P = S + (BORN ? B3_P / 2 : G3_P) * plane;
    const R *br = BORN ? reinterpret_cast<const R *>(a.br2) : reinterpret_cast<const R *>(a.binv);
    const int shot = a.shot0 + c.slot;
    const long long bandoff = band_base(a.bands, shot, a.n);
    const float dt = g.dt;
    const R b0 = br[cc];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int i = coord(c, d), N = extent(g, d);
        const long long sd = stride(g, d);
        const float *cd = cdir(g, d);
        T G = diff<M, T>(cd, [&](int l) {
            T a1 = (i + l < N) ? P[cc + l * sd] : zero_<T>();
            T b1 = (i + 1 - l >= 0) ? P[cc + (1 - l) * sd] : zero_<T>();
            return sub_(a1, b1);
        });
        if (pml_half(g, d, i)) {
            T *ps = S + (BORN ? (B3_PP + 2 * d) / 2 : G3_PP + d) * plane;
            T v = fma_(a.pml.bh[d][i], ps[cc], mul_(a.pml.ah[d][i], G));
            ps[cc] = v;
            G = add_(G, v);
        }
        const R b1 = (i + 1 < N) ? br[cc + sd] : b0;
        const float bu = 0.5f * (xof(b0) + xof(b1));
        T *V = S + (BORN ? (B3_V + 2 * d) / 2 : G3_V + d) * plane;
        T vn = fma_(-dt * bu, G, V[cc]);
        if constexpr (BORN) {
            const float rs = yof(b0) + ((i + 1 < N) ? yof(b1) : 0.f);
            vn.y = fmaf(0.5f * dt * rs, G.x, vn.y);
        }
        V[cc] = vn;
        if (BANDS) {
            long long b = face_band(g, d, c.z - g.z0, c.y - g.y0, c.x - g.x0);
            if (b >= 0) band_put(a.bands, 1, c.slot, bandoff, b, xof(vn));
        }
        if (HESS) {
            float q = bu * xof(G);
            st[(G3_HQ + d) * plane + cc] = q * q;
        }
    }
}

// ---------------------------------------------------------------------------
// Forward pressure stage (nodes), in place: source, Born records, p band.
// ---------------------------------------------------------------------------
template <int M, bool BORN, bool BANDS, bool HESS>
__global__ void __launch_bounds__(256) k3_p(const Step3D a)
{
    using T = typename std::conditional<BORN, float2, float>::type;
    using K = typename std::conditional<BORN, float2, float>::type;
    const GridDev &g = a.g;
    const Cell c = cell_of(g);
    if (!c.ok) return;
    const long long plane = g.plane;
    const long long cc = (long long)c.z * g.rowz + (long long)c.y * g.pitch + c.x;
    float *st = a.st + c.slot * a.sstride;
    T *S = reinterpret_cast<T *>(st);
    const int shot = a.shot0 + c.slot;
    const float dt = g.dt;
    T Q = zero_<T>();
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int i = coord(c, d), N = extent(g, d);
        const long long sd = stride(g, d);
        const T *V = S + (BORN ? (B3_V + 2 * d) / 2 : G3_V + d) * plane;
        T q = diff<M, T>(cdir(g, d), [&](int l) {
            T a1 = (i + l - 1 < N) ? V[cc + (l - 1) * sd] : zero_<T>();
            T b1 = (i - l >= 0) ? V[cc - l * sd] : zero_<T>();
            return sub_(a1, b1);
        });
        if (pml_node(g, d, i)) {
            T *pv = S + (BORN ? (B3_PV + 2 * d) / 2 : G3_PV + d) * plane;
            T v = fma_(a.pml.bi[d][i], pv[cc], mul_(a.pml.ai[d][i], q));
            pv[cc] = v;
            q = add_(q, v);
        }
        Q = add_(Q, q);
    }
    T *P = S + (BORN ? B3_P / 2 : G3_P) * plane;
    const T p0 = P[cc];
    const K kd2 = BORN ? reinterpret_cast<const K *>(a.kd2)[cc] : reinterpret_cast<const K *>(a.kdt)[cc];
    const float kd = xof(kd2);
    T pn = fma_(-kd, Q, p0);
    if constexpr (BORN) pn.y = fmaf(-yof(kd2), Q.x, pn.y);
    if (cc == a.src_cell[shot]) {
        const float w = a.src_scale * a.wav[(a.wav_per_shot ? (long long)shot * g.nt : 0) + a.n];
        if constexpr (BORN) pn.x += w;
        else pn += w;
    }
    P[cc] = pn;
    const int iz = c.z - g.z0, iy = c.y - g.y0, ix = c.x - g.x0;
    if (BANDS) {
        long long b = pband3(g, iz, iy, ix);
        if (b >= 0) band_put(a.bands, 0, c.slot, band_base(a.bands, shot, a.n), b, xof(p0));
    }
    if (HESS) {
        if (iz >= 0 && iz < g.nz && iy >= 0 && iy < g.ny && ix >= 0 && ix < g.nx) {
            float hr = 0.f;
            for (int d = 0; d < 3; ++d) {
                const float *hq = st + (G3_HQ + d) * plane;
                hr += hq[cc] + hq[cc - stride(g, d)];
            }
            const float bi = a.binv[cc];
            const float kq = kd * xof(Q) / dt;
            a.hess[c.slot * plane + cc] += dt * (0.5f * hr / (bi * bi) + kq * kq);
        }
    }
    if (BORN || a.rec_bg) {
        // record dp^{n+1} (Born) or the background p^{n+1} (nonlinear modelling)
        const int k = a.rmap[(long long)shot * plane + cc];
        if (k >= 0) {
            float v;
            if constexpr (BORN) v = a.rec_bg ? xof(pn) : yof(pn);
            else v = xof(pn);
            const int e = a.rptr[shot + 1];
            for (int q = k; q < e && a.rcell[q] == cc; ++q)
                a.dstage[(long long)a.rrow[q] * g.nt + a.n] = v;
        }
    }
}

// Residual of step n at node cc of shot `shot` (sum over the receivers there).
__device__ __forceinline__ float residual_at(const Step3D &a, int shot, long long cc, int n)
{
    const int k = a.rmap[(long long)shot * a.g.plane + cc];
    if (k < 0) return 0.f;
    float add = 0.f;
    const int e = a.rptr[shot + 1];
    for (int q = k; q < e && a.rcell[q] == cc; ++q) add += a.dstage[(long long)a.rrow[q] * a.g.nt + n];
    return add;
}

__device__ __forceinline__ bool interior(const GridDev &g, const Cell &c)
{
    const int iz = c.z - g.z0, iy = c.y - g.y0, ix = c.x - g.x0;
    return iz >= 0 && iz < g.nz && iy >= 0 && iy < g.ny && ix >= 0 && ix < g.nx;
}

// ---------------------------------------------------------------------------
// Reverse start (step nt-1): lambda_p = R^T d_{nt-1}, kappa image of step
// nt-1 from Q = D- . v^{nt-1/2}.
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(256) k3_adj_init(const Step3D a)
{
    const GridDev &g = a.g;
    const Cell c = cell_of(g);
    if (!c.ok) return;
    const long long plane = g.plane;
    const long long cc = (long long)c.z * g.rowz + (long long)c.y * g.pitch + c.x;
    float *st = a.st + c.slot * a.sstride;
    float2 *S = reinterpret_cast<float2 *>(st);
    const int shot = a.shot0 + c.slot;
    const float lp1 = residual_at(a, shot, cc, g.nt - 1);
    S[(A3_PL / 2) * plane + cc].y = a.kdt[cc] * lp1;   // mu
    if (interior(g, c)) {
        float Q = 0.f;
        for (int d = 0; d < 3; ++d) {
            const int i = coord(c, d), N = extent(g, d);
            const long long sd = stride(g, d);
            const float2 *V = S + ((A3_V + 2 * d) / 2) * plane;
            Q += diff<M, float>(cdir(g, d), [&](int l) {
                float a1 = (i + l - 1 < N) ? V[cc + (l - 1) * sd].x : 0.f;
                float b1 = (i - l >= 0) ? V[cc - l * sd].x : 0.f;
                return a1 - b1;
            });
        }
        st[A3_IMK * plane + cc] += Q * lp1;
    }
}

// ---------------------------------------------------------------------------
// Reverse half-node stage of step n: S4^T/S3^T (lambda_v from lambda_p),
// lambda_psi_p of S2^T, background v^{n-1/2}, rho-image products.
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(256) k3_a(const Step3D a)
{
    const GridDev &g = a.g;
    const Cell c = cell_of(g);
    if (!c.ok) return;
    const long long plane = g.plane;
    const long long cc = (long long)c.z * g.rowz + (long long)c.y * g.pitch + c.x;
    float *st = a.st + c.slot * a.sstride;
    float2 *S = reinterpret_cast<float2 *>(st);
    const float2 *PL = S + (A3_PL / 2) * plane;
    const int shot = a.shot0 + c.slot;
    const float dt = g.dt;
    const bool recon = a.n > 0;
    const long long rowprev = band_row(a.bands, shot, a.n - 1);
    const float b0 = a.binv[cc];
    const int iz = c.z - g.z0, iy = c.y - g.y0, ix = c.x - g.x0;
    for (int d = 0; d < 3; ++d) {
        const int i = coord(c, d), N = extent(g, d);
        const long long sd = stride(g, d);
        const float *lpv = st + (A3_LPV + d) * plane;
        // (p^n, kdt*lp - ai_d (lpsi_vd - kdt*lp)) at a node along d
        auto pu = [&](int j, long long cj) -> float2 {
            if (j < 0 || j >= N) return make_float2(0.f, 0.f);
            const float2 pl = PL[cj];   // (p, mu)
            float u = pl.y;
            if (pml_node(g, d, j)) u -= a.pml.ai[d][j] * (lpv[cj] - pl.y);
            return make_float2(pl.x, u);
        };
        const float2 D = diff<M, float2>(cdir(g, d), [&](int l) {
            return sub_(pu(i + l, cc + l * sd), pu(i + 1 - l, cc + (1 - l) * sd));
        });   // (G_d, du/dd)
        float2 *V = S + ((A3_V + 2 * d) / 2) * plane;
        const float2 v = V[cc];   // (v, w)
        const float b1 = (i + 1 < N) ? a.binv[cc + sd] : b0;
        const float dtbu = dt * 0.5f * (b0 + b1);
        const float lv = v.y / dtbu + D.y;
        if (pml_half(g, d, i)) {
            float *lpp = st + (A3_LPP + d) * plane;
            lpp[cc] = a.pml.bh[d][i] * lpp[cc] - dtbu * lv;
        }
        st[(A3_IM + d) * plane + cc] += D.x * lv;
        float vn = 0.f;
        if (recon) {
            bool inner_h = iz >= 0 && iz < g.nz && iy >= 0 && iy < g.ny && ix >= 0 && ix < g.nx;
            if (inner_h) vn = v.x + dtbu * D.x;
            else {
                long long b = face_band(g, d, iz, iy, ix);
                if (b >= 0) vn = band_get(a.bands, 1, rowprev, b);
            }
        }
        V[cc] = make_float2(vn, dtbu * lv);
    }
}

// ---------------------------------------------------------------------------
// Reverse node stage of step n >= 1: S2^T/S1^T (lambda_p from lambda_v and
// lambda_psi_p), lambda_psi_v, background p^{n-1}, injection of the residual
// of step n-1 and the kappa image of step n-1.
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(256) k3_b(const Step3D a)
{
    const GridDev &g = a.g;
    const Cell c = cell_of(g);
    if (!c.ok) return;
    const long long plane = g.plane;
    const long long cc = (long long)c.z * g.rowz + (long long)c.y * g.pitch + c.x;
    float *st = a.st + c.slot * a.sstride;
    float2 *S = reinterpret_cast<float2 *>(st);
    const int shot = a.shot0 + c.slot;
    const int n = a.n;
    float2 *PL = S + (A3_PL / 2) * plane;
    const float2 pl = PL[cc];   // (p, mu)
    const float kd = a.kdt[cc];
    const float lp = pl.y / kd;
    float2 E = make_float2(0.f, 0.f);   // (D- . v^{n-1/2}, D- . w)
    for (int d = 0; d < 3; ++d) {
        const int i = coord(c, d), N = extent(g, d);
        const long long sd = stride(g, d);
        const float2 *V = S + ((A3_V + 2 * d) / 2) * plane;
        const float *lpp = st + (A3_LPP + d) * plane;
        // (v^{n-1/2}, dt bu lambda_v - ah lambda_psi_p) at a half node along d
        auto vw = [&](int j, long long cj) -> float2 {
            if (j < 0 || j >= N) return make_float2(0.f, 0.f);
            const float2 v = V[cj];   // (v, w)
            float w = v.y;
            if (pml_half(g, d, j)) w -= a.pml.ah[d][j] * lpp[cj];
            return make_float2(v.x, w);
        };
        E = add_(E, diff<M, float2>(cdir(g, d), [&](int l) {
                     return sub_(vw(i + l - 1, cc + (l - 1) * sd), vw(i - l, cc - l * sd));
                 }));
        if (pml_node(g, d, i)) {
            float *lpv = st + (A3_LPV + d) * plane;
            lpv[cc] = a.pml.bi[d][i] * (lpv[cc] - pl.y);
        }
    }
    const float lp3 = lp + E.y;
    const bool in = interior(g, c);
    float pn = 0.f;
    if (in) {
        pn = pl.x + kd * E.x;
        if (cc == a.src_cell[shot])
            pn -= a.src_scale * a.wav[(a.wav_per_shot ? (long long)shot * g.nt : 0) + n - 1];
    } else {
        long long b = pband3(g, c.z - g.z0, c.y - g.y0, c.x - g.x0);
        if (b >= 0) pn = band_get(a.bands, 0, band_row(a.bands, shot, n - 1), b);
    }
    const float lpn = lp3 + residual_at(a, shot, cc, n - 1);
    if (in) st[A3_IMK * plane + cc] += E.x * lpn;
    PL[cc] = make_float2(pn, kd * lpn);
}

// lambda_psi_p memories hold S2^T values before the b_h scaling of S1^T; the
// half-node stage of the next step applies b_h to them (k3_a reads
// bh * stored - dt bu lambda_v).

// Adjoint start state (p, 0), (v_x, 0), (v_y, 0), (v_z, 0) from the saved
// background final state [p][vx][vy][vz].
__global__ void k3_pack(const GridDev g, const float *final_state, int shot0, int batch, float *st,
                        long long sstride)
{
    const long long plane = g.plane;
    const long long n = batch * plane;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long s = i / plane, c = i - s * plane;
        const float *fs = final_state + (shot0 + s) * 4 * plane;
        float2 *o = reinterpret_cast<float2 *>(st + s * sstride);
        o[(A3_PL / 2) * plane + c] = make_float2(fs[c], 0.f);
        for (int d = 0; d < 3; ++d) o[((A3_V + 2 * d) / 2) * plane + c] = make_float2(fs[(1 + d) * plane + c], 0.f);
    }
}

// Per-batch stacking: acc.x += sum_slots kappa image, acc.y += sum_slots
// sum_d (half-node product at the node + at the node - e_d).
__global__ void k3_image_acc(const GridDev g, const float *st, long long sstride, int batch, double2 *acc)
{
    const long long nint = (long long)g.nz * g.ny * g.nx;
    const long long plane = g.plane;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nint;
         k += (long long)gridDim.x * blockDim.x) {
        const long long ix = k % g.nx, t = k / g.nx, iy = t % g.ny, iz = t / g.ny;
        const long long c = (iz + g.z0) * g.rowz + (iy + g.y0) * g.pitch + (ix + g.x0);
        double2 s = acc[k];
        for (int b = 0; b < batch; ++b) {
            const float *sl = st + b * sstride;
            s.x += sl[A3_IMK * plane + c];
            double r = 0.0;
            for (int d = 0; d < 3; ++d) {
                const long long sd = d == 0 ? g.rowz : (d == 1 ? (long long)g.pitch : 1LL);
                r += (double)sl[(A3_IM + d) * plane + c] + (double)sl[(A3_IM + d) * plane + c - sd];
            }
            s.y += r;
        }
        acc[k] = s;
    }
}

dim3 grid3(const GridDev &g, int batch) { return dim3((g.Nx + 31) / 32, (g.Ny + 7) / 8, g.Nz * batch); }

}  // namespace

cudaError_t launch_fwd3d(const Step3D &a, int batch, bool born, bool bands, bool hess, int stages,
                         cudaStream_t s)
{
    const dim3 blk(32, 8), grd = grid3(a.g, batch);
#define L3(MM, B, BA, H)                                                  \
    do {                                                                  \
        if (stages & 1) k3_v<MM, B, BA, H><<<grd, blk, 0, s>>>(a);        \
        if (stages & 2) k3_p<MM, B, BA, H><<<grd, blk, 0, s>>>(a);        \
    } while (0)
    if (a.g.M == 2) {
        if (born) L3(2, true, false, false);
        else if (bands && hess) L3(2, false, true, true);
        else if (bands) L3(2, false, true, false);
        else if (hess) L3(2, false, false, true);
        else L3(2, false, false, false);
    } else {
        if (born) L3(4, true, false, false);
        else if (bands && hess) L3(4, false, true, true);
        else if (bands) L3(4, false, true, false);
        else if (hess) L3(4, false, false, true);
        else L3(4, false, false, false);
    }
#undef L3
    return cudaGetLastError();
}

cudaError_t launch_adj3d_init(const Step3D &a, int batch, cudaStream_t s)
{
    const dim3 blk(32, 8), grd = grid3(a.g, batch);
    if (a.g.M == 2) k3_adj_init<2><<<grd, blk, 0, s>>>(a);
    else k3_adj_init<4><<<grd, blk, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adj3d(const Step3D &a, int batch, cudaStream_t s)
{
    const dim3 blk(32, 8), grd = grid3(a.g, batch);
    if (a.g.M == 2) {
        k3_a<2><<<grd, blk, 0, s>>>(a);
        if (a.n > 0) k3_b<2><<<grd, blk, 0, s>>>(a);
    } else {
        k3_a<4><<<grd, blk, 0, s>>>(a);
        if (a.n > 0) k3_b<4><<<grd, blk, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_adjoint3d(const GridDev &g, const float *final_state, int shot0, int batch, float *st,
                                  long long sstride, cudaStream_t s)
{
    long long n = batch * g.plane;
    int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 16);
    k3_pack<<<blocks, 256, 0, s>>>(g, final_state, shot0, batch, st, sstride);
    return cudaGetLastError();
}

cudaError_t launch_image_accumulate3d(const GridDev &g, const float *st, long long sstride, int batch,
                                      double2 *acc, cudaStream_t s)
{
    long long n = (long long)g.nz * g.ny * g.nx;
    int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 16);
    k3_image_acc<<<blocks, 256, 0, s>>>(g, st, sstride, batch, acc);
    return cudaGetLastError();
}

}  // namespace lsrtm
