// 3D background time-step kernels (Eq. 1): the forward pass that saves the
// boundary bands and the final state for the reverse reconstruction (App. A),
// accumulates the pseudo-Hessian diagonal (App. B), records the pressure for
// nonlinear modelling, and recomputes band segments in checkpoint mode.
//
// Each time step is two launches over all shots of a batch, one thread per
// padded cell, updating the state in place: k3_v (half nodes: v_x, v_y, v_z
// and their CPML memories from D+ p) then k3_p (nodes: p from D- . v,
// source, records, bands). These passes run once per solve (their bands are
// cached across L^T calls); the Born operator and its transpose, which every
// CG iteration repeats, use the fused kernels of kernels3d_fused.cu.
#include <algorithm>

#include "lsrtm_internal.cuh"

namespace lsrtm {
namespace {

// Slot layout in float planes (state updated in place), d = 0 z, 1 y, 2 x:
// p | v_d | psi_p,d | psi_v,d | (bu G_d)^2.
enum { G3_P = 0, G3_V = 1, G3_PP = 4, G3_PV = 7, G3_HQ = 10 };   // + d


template <int M, class T, class F>
__device__ __forceinline__ T diff(const float *c, F f)   // sum_l c_l (f(l) - f(1 - l)) as (a_l, b_l) pairs
{
    T d[M];
#pragma unroll
    for (int l = 0; l < M; ++l) d[l] = f(l + 1);
    T acc = c[0] * d[0];
#pragma unroll
    for (int l = 1; l < M; ++l) acc = fmaf(c[l], d[l], acc);
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
template <int M, bool BANDS, bool HESS>
__global__ void __launch_bounds__(256) k3_v(const Step3D a)
{
    if (guard_tripped(a.g)) return;
    const GridDev &g = a.g;
    const Cell c = cell_of(g);
    if (!c.ok) return;
    const long long plane = g.plane;
    const long long cc = (long long)c.z * g.rowz + (long long)c.y * g.pitch + c.x;
    float *st = a.st + c.slot * a.sstride;
    const float *P = st + G3_P * plane;
    const float *br = a.binv;
    const int shot = a.shot0 + c.slot;
    const long long bandoff = band_base(a.bands, shot, a.n);
    const float dt = g.dt;
    const float b0 = br[cc];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int i = coord(c, d), N = extent(g, d);
        const long long sd = stride(g, d);
        // p at node row j along d (free surface: a ghost z row holds -p(mirror))
        auto pj = [&](int j) -> float {
            if (j < 0 || j >= N) return 0.f;
            if (d == 0 && g.fs && j < g.z0) return -P[cc + (long long)(fs_node_row(g, j) - i) * sd];
            return P[cc + (long long)(j - i) * sd];
        };
        float G = diff<M, float>(cdir(g, d), [&](int l) { return pj(i + l) - pj(i + 1 - l); });
        if (pml_half(g, d, i)) {
            float *ps = st + (G3_PP + d) * plane;
            const float v = fmaf(a.pml.bh[d][i], ps[cc], a.pml.ah[d][i] * G);
            ps[cc] = v;
            G += v;
        }
        const float b1 = (i + 1 < N) ? br[cc + sd] : b0;
        const float bu = 0.5f * (b0 + b1);
        float *V = st + (G3_V + d) * plane;
        const float vn = fmaf(-dt * bu, G, V[cc]);
        V[cc] = vn;
        if (BANDS) {
            const long long b = face_band(g, d, c.z - g.z0, c.y - g.y0, c.x - g.x0);
            if (b >= 0) band_put(a.bands, 1, c.slot, bandoff, b, vn);
        }
        if (HESS) {
            const float q = bu * G;
            st[(G3_HQ + d) * plane + cc] = q * q;
        }
    }
}

// ---------------------------------------------------------------------------
// Forward pressure stage (nodes), in place: source, p band, pseudo-Hessian,
// pressure records (nonlinear modelling).
// ---------------------------------------------------------------------------
template <int M, bool BANDS, bool HESS>
__global__ void __launch_bounds__(256) k3_p(const Step3D a)
{
    if (guard_tripped(a.g)) return;
    const GridDev &g = a.g;
    const Cell c = cell_of(g);
    if (!c.ok) return;
    const long long plane = g.plane;
    const long long cc = (long long)c.z * g.rowz + (long long)c.y * g.pitch + c.x;
    float *st = a.st + c.slot * a.sstride;
    const int shot = a.shot0 + c.slot;
    const float dt = g.dt;
    // D- . v summed z, y, x (the reverse reconstruction sums in the same order)
    float Q = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int i = coord(c, d), N = extent(g, d);
        const long long sd = stride(g, d);
        const float *V = st + (G3_V + d) * plane;
        // v_d at half row j along d (free surface: a ghost z half row holds v_z(mirror))
        auto vj = [&](int j) -> float {
            if (j < 0 || j >= N) return 0.f;
            if (d == 0 && g.fs && j < g.z0) return V[cc + (long long)(fs_half_row(g, j) - i) * sd];
            return V[cc + (long long)(j - i) * sd];
        };
        float q = diff<M, float>(cdir(g, d), [&](int l) { return vj(i + l - 1) - vj(i - l); });
        if (pml_node(g, d, i)) {
            float *pv = st + (G3_PV + d) * plane;
            const float v = fmaf(a.pml.bi[d][i], pv[cc], a.pml.ai[d][i] * q);
            pv[cc] = v;
            q += v;
        }
        Q += q;
    }
    float *P = st + G3_P * plane;
    const float p0 = P[cc];
    const float kd = a.kdt[cc];
    float pn = fmaf(-kd, Q, p0);
    if (cc == a.src_cell[shot]) pn += a.src_scale * a.wav[(a.wav_per_shot ? (long long)shot * g.nt : 0) + a.n];
    if (g.fs && c.z <= g.z0) pn = 0.f;   // p = 0 on the free surface (ghost rows unused)
    P[cc] = pn;
    const int iz = c.z - g.z0, iy = c.y - g.y0, ix = c.x - g.x0;
    if (BANDS) {
        const long long b = pband3(g, iz, iy, ix);
        if (b >= 0) band_put(a.bands, 0, c.slot, band_base(a.bands, shot, a.n), b, p0);
    }
    if (HESS) {
        if (iz >= 0 && iz < g.nz && iy >= 0 && iy < g.ny && ix >= 0 && ix < g.nx) {
            float hr = 0.f;
            for (int d = 0; d < 3; ++d) {
                const float *hq = st + (G3_HQ + d) * plane;
                hr += hq[cc] + hq[cc - stride(g, d)];
            }
            const float bi = a.binv[cc];
            const float kq = kd * Q / dt;
            a.hess[c.slot * plane + cc] += dt * (0.5f * hr / (bi * bi) + kq * kq);
        }
    }
    if (a.rec_bg) {
        // record the pressure p^{n+1} (nonlinear modelling)
        const int k = a.rmap[(long long)shot * plane + cc];
        if (k >= 0) {
            const int e = a.rptr[shot + 1];
            for (int q = k; q < e && a.rcell[q] == cc; ++q) a.dstage[(long long)a.rrow[q] * g.nt + a.n] = pn;
        }
    }
}

dim3 grid3(const GridDev &g, int batch) { return dim3((g.Nx + 31) / 32, (g.Ny + 7) / 8, g.Nz * batch); }

}  // namespace

cudaError_t launch_fwd3d(const Step3D &a, int batch, bool bands, bool hess, int stages, cudaStream_t s)
{
    const dim3 blk(32, 8), grd = grid3(a.g, batch);
#define L3(MM, BA, H)                                                  \
    do {                                                               \
        if (stages & 1) k3_v<MM, BA, H><<<grd, blk, 0, s>>>(a);        \
        if (stages & 2) k3_p<MM, BA, H><<<grd, blk, 0, s>>>(a);        \
    } while (0)
    if (a.g.M == 2) {
        if (bands && hess) L3(2, true, true);
        else if (bands) L3(2, true, false);
        else if (hess) L3(2, false, true);
        else L3(2, false, false);
    } else {
        if (bands && hess) L3(4, true, true);
        else if (bands) L3(4, true, false);
        else if (hess) L3(4, false, true);
        else L3(4, false, false);
    }
#undef L3
    return cudaGetLastError();
}

}  // namespace lsrtm
