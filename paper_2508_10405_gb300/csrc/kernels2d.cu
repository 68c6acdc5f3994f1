// Fused 2D time-step kernels for the staggered-grid Born operator and its
// exact transpose (Eq. 1, Eq. scattereqln, App. A).
//
// One launch advances every shot of a batch by one time step. A CTA owns a
// TZ x TX tile of integer nodes. It stages the pressure fields on the tile
// plus a (2M-1)-deep halo in shared memory, recomputes the velocity stage on
// the tile plus an M-deep halo (redundantly with its neighbours, so no grid
// barrier is needed between the v and p stages), then finishes the pressure
// stage on its own tile. Each state field is therefore read once and written
// once per step; the halo reads are served by L2. Inputs and outputs are
// separate (ping-pong) buffers, so neighbouring CTAs never race.
#include "lsrtm_internal.cuh"

namespace lsrtm {
namespace {

constexpr int TX = kTX2;
constexpr int TZ = kTZ2;
constexpr int NTH = kThreads2D;

// Field planes of a shot slot.
// Forward (background + Born): p vx vz psi_px psi_pz | dp dvx dvz dpsi_px dpsi_pz;
// node CPML memories in place: psi_vx psi_vz dpsi_vx dpsi_vz.
enum { F_P = 0, F_VX = 1, F_VZ = 2, F_PPX = 3, F_PPZ = 4, F_D = 5 };
// Adjoint: background p vx vz | lambda p vx vz | lambda psi_px psi_pz psi_vx psi_vz.
enum { A_P = 0, A_VX = 1, A_VZ = 2, A_LP = 3, A_LVX = 4, A_LVZ = 5, A_LPPX = 6, A_LPPZ = 7,
       A_LPVX = 8, A_LPVZ = 9 };

template <int M>
struct Geo {
    static constexpr int H = 2 * M - 1;            // pressure halo depth
    static constexpr int HX = (H + 3) & ~3;         // x halo rounded for float4 loads
    static constexpr int SX = TX + 2 * HX;
    static constexpr int SZ = TZ + 2 * H;
    static constexpr int VXW = TX + 2 * M;          // x half nodes [tx0-M, tx0+TX+M-1)
    static constexpr int VZH = TZ + 2 * M;          // z half rows  [tz0-M, tz0+TZ+M-1)
    static constexpr int NVX = TZ * (VXW - 1);
    static constexpr int NVZ = (VZH - 1) * TX;
};

__device__ __forceinline__ long long band_xstrip(int iz, int ix, int M, int nz, int nx)
{
    return ix < 0 ? (long long)iz * M + (ix + M) : (long long)M * nz + (long long)iz * M + (ix - nx);
}

__device__ __forceinline__ long long band_zstrip(int iz, int ix, int M, int nz, int nx)
{
    long long base = 2LL * M * nz;
    return iz < 0 ? base + (long long)(iz + M) * nx + ix
                  : base + (long long)M * nx + (long long)(iz - nz) * nx + ix;
}

// Band slot of a node for the p band, -1 if the node is not in it.
__device__ __forceinline__ long long pband_index(int iz, int ix, int M, int nz, int nx)
{
    if (iz >= 0 && iz < nz) {
        if ((ix >= -M && ix < 0) || (ix >= nx && ix < nx + M)) return band_xstrip(iz, ix, M, nz, nx);
        return -1;
    }
    if (ix >= 0 && ix < nx && ((iz >= -M && iz < 0) || (iz >= nz && iz < nz + M)))
        return band_zstrip(iz, ix, M, nz, nx);
    return -1;
}

__device__ __forceinline__ void band_put(const Bands &b, void *base, long long off, float v)
{
    if (b.bf16) reinterpret_cast<__nv_bfloat16 *>(base)[off] = __float2bfloat16_rn(v);
    else reinterpret_cast<float *>(base)[off] = v;
}

__device__ __forceinline__ float band_get(const Bands &b, const void *base, long long off)
{
    if (b.bf16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(base)[off]);
    return reinterpret_cast<const float *>(base)[off];
}

// Loads a (SZ x SX) box of one field starting at (tz0-H, tx0-HX) with 128-bit
// loads; cells outside the padded array read as zero.
template <int M>
__device__ __forceinline__ void load_box(float *dst, const float *src, const GridDev &g, int tz0,
                                         int tx0)
{
    using G = Geo<M>;
    constexpr int SX4 = G::SX / 4;
    for (int i = threadIdx.x; i < G::SZ * SX4; i += NTH) {
        int rz = i / SX4, q = i - rz * SX4;
        int z = tz0 - G::H + rz, x = tx0 - G::HX + 4 * q;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (z >= 0 && z < g.Nz && x >= 0 && x < g.pitch)
            v = __ldg(reinterpret_cast<const float4 *>(src + (long long)z * g.pitch + x));
        *reinterpret_cast<float4 *>(dst + rz * G::SX + 4 * q) = v;
    }
}

// ---------------------------------------------------------------------------
// Forward step: background (and, if BORN, the scattered field) from step n to
// n+1. BANDS saves the boundary bands of p^n and v^{n+1/2}; HESS accumulates
// the pseudo-Hessian diagonal of App. B.
// ---------------------------------------------------------------------------
template <int M, bool BORN, bool BANDS, bool HESS>
__global__ void __launch_bounds__(NTH) k_fwd2d(const Step2D a)
{
    using G = Geo<M>;
    constexpr int NF = BORN ? 2 : 1;
    constexpr int H = G::H, HX = G::HX, SX = G::SX, SZ = G::SZ, VXW = G::VXW;
    extern __shared__ __align__(16) float smem[];
    float *sP = smem;                       // [NF][SZ][SX]
    float *sVx = sP + NF * SZ * SX;         // [NF][TZ][VXW]
    float *sVz = sVx + NF * TZ * VXW;       // [NF][VZH][TX]
    float *sHx = sVz + NF * G::VZH * TX;    // [TZ][TX+1]
    float *sHz = sHx + TZ * (TX + 1);       // [TZ+1][TX]

    const GridDev &g = a.g;
    const int tid = threadIdx.x;
    const int tx0 = blockIdx.x * TX, tz0 = blockIdx.y * TZ;
    const int slot = blockIdx.z, shot = a.shot0 + slot;
    const int pitch = g.pitch;
    const long long plane = g.plane;
    const float *in = a.in + slot * a.sstride;
    float *out = a.out + slot * a.sstride;
    float *psiv = a.psiv + slot * a.vstride;
    const float dt = g.dt;
    const int x0 = g.x0, x1 = g.x0 + g.nx, z0 = g.z0, z1 = g.z0 + g.nz;
    const long long bandoff = ((long long)shot * g.nt + a.n) * a.bands.nb;

    load_box<M>(sP, in + F_P * plane, g, tz0, tx0);
    if (BORN) load_box<M>(sP + SZ * SX, in + (F_D + F_P) * plane, g, tz0, tx0);
    __syncthreads();

    // ---- velocity stage along x on the tile + M halo
    for (int i = tid; i < G::NVX; i += NTH) {
        int r = i / (VXW - 1), ci = i - r * (VXW - 1);
        int z = tz0 + r, j = tx0 - M + ci;
        float vn = 0.f, dvn = 0.f, hq = 0.f;
        if (z < g.Nz && j >= 0 && j < g.Nx) {
            const float *pr = sP + (r + H) * SX + (ci - M + HX);
            float dp = 0.f;
#pragma unroll
            for (int l = 1; l <= M; ++l) dp += g.cx[l - 1] * (pr[l] - pr[1 - l]);
            long long cell = (long long)z * pitch + j;
            bool own = ci >= M && ci < M + TX;
            bool pml = (j <= x0 - 2) || (j >= x1);
            float Gx = dp;
            if (pml) {
                float ps = a.pml.bh[2][j] * __ldg(in + F_PPX * plane + cell) + a.pml.ah[2][j] * dp;
                Gx += ps;
                if (own) out[F_PPX * plane + cell] = ps;
            }
            float bu = 0.5f * (__ldg(a.binv + cell) + __ldg(a.binv + (j + 1 < g.Nx ? cell + 1 : cell)));
            float dtbu = dt * bu;
            vn = __ldg(in + F_VX * plane + cell) - dtbu * Gx;
            if (BORN) {
                const float *dr = pr + SZ * SX;
                float ddp = 0.f;
#pragma unroll
                for (int l = 1; l <= M; ++l) ddp += g.cx[l - 1] * (dr[l] - dr[1 - l]);
                float Gd = ddp;
                if (pml) {
                    float ps = a.pml.bh[2][j] * __ldg(in + (F_D + F_PPX) * plane + cell) +
                               a.pml.ah[2][j] * ddp;
                    Gd += ps;
                    if (own) out[(F_D + F_PPX) * plane + cell] = ps;
                }
                float r0 = __ldg(a.rr + cell), r1 = (j + 1 < g.Nx) ? __ldg(a.rr + cell + 1) : 0.f;
                float dtdbu = -0.5f * dt * (r0 + r1);
                dvn = __ldg(in + (F_D + F_VX) * plane + cell) - dtbu * Gd - dtdbu * Gx;
            }
            if (own) {
                out[F_VX * plane + cell] = vn;
                if (BORN) out[(F_D + F_VX) * plane + cell] = dvn;
                if (BANDS) {
                    int iz = z - z0, ix = j - x0;
                    if (iz >= 0 && iz < g.nz && ((ix >= -M && ix < 0) || (ix >= g.nx && ix < g.nx + M)))
                        band_put(a.bands, a.bands.v, bandoff + band_xstrip(iz, ix, M, g.nz, g.nx), vn);
                }
            }
            if (HESS) { float t = bu * Gx; hq = t * t; }
        }
        sVx[r * VXW + ci] = vn;
        if (BORN) sVx[TZ * VXW + r * VXW + ci] = dvn;
        if (HESS && ci >= M - 1 && ci < M + TX) sHx[r * (TX + 1) + (ci - M + 1)] = hq;
    }
    // ---- velocity stage along z on the tile + M halo
    for (int i = tid; i < G::NVZ; i += NTH) {
        int r = i / TX, c = i - r * TX;
        int k = tz0 - M + r, x = tx0 + c;
        float vn = 0.f, dvn = 0.f, hq = 0.f;
        if (k >= 0 && k < g.Nz && x < g.Nx) {
            const float *pc = sP + (r - M + H) * SX + (c + HX);
            float dp = 0.f;
#pragma unroll
            for (int l = 1; l <= M; ++l) dp += g.cz[l - 1] * (pc[l * SX] - pc[(1 - l) * SX]);
            long long cell = (long long)k * pitch + x;
            bool own = r >= M && r < M + TZ;
            bool pml = (k <= z0 - 2) || (k >= z1);
            float Gz = dp;
            if (pml) {
                float ps = a.pml.bh[0][k] * __ldg(in + F_PPZ * plane + cell) + a.pml.ah[0][k] * dp;
                Gz += ps;
                if (own) out[F_PPZ * plane + cell] = ps;
            }
            float bu = 0.5f * (__ldg(a.binv + cell) + __ldg(a.binv + (k + 1 < g.Nz ? cell + pitch : cell)));
            float dtbu = dt * bu;
            vn = __ldg(in + F_VZ * plane + cell) - dtbu * Gz;
            if (BORN) {
                const float *dc = pc + SZ * SX;
                float ddp = 0.f;
#pragma unroll
                for (int l = 1; l <= M; ++l) ddp += g.cz[l - 1] * (dc[l * SX] - dc[(1 - l) * SX]);
                float Gd = ddp;
                if (pml) {
                    float ps = a.pml.bh[0][k] * __ldg(in + (F_D + F_PPZ) * plane + cell) +
                               a.pml.ah[0][k] * ddp;
                    Gd += ps;
                    if (own) out[(F_D + F_PPZ) * plane + cell] = ps;
                }
                float r0 = __ldg(a.rr + cell), r1 = (k + 1 < g.Nz) ? __ldg(a.rr + cell + pitch) : 0.f;
                float dtdbu = -0.5f * dt * (r0 + r1);
                dvn = __ldg(in + (F_D + F_VZ) * plane + cell) - dtbu * Gd - dtdbu * Gz;
            }
            if (own) {
                out[F_VZ * plane + cell] = vn;
                if (BORN) out[(F_D + F_VZ) * plane + cell] = dvn;
                if (BANDS) {
                    int iz = k - z0, ix = x - x0;
                    if (ix >= 0 && ix < g.nx && ((iz >= -M && iz < 0) || (iz >= g.nz && iz < g.nz + M)))
                        band_put(a.bands, a.bands.v, bandoff + band_zstrip(iz, ix, M, g.nz, g.nx), vn);
                }
            }
            if (HESS) { float t = bu * Gz; hq = t * t; }
        }
        sVz[r * TX + c] = vn;
        if (BORN) sVz[G::VZH * TX + r * TX + c] = dvn;
        if (HESS && r >= M - 1 && r < M + TZ) sHz[(r - M + 1) * TX + c] = hq;
    }
    __syncthreads();

    // ---- pressure stage on the own tile
    const int src = a.src_cell[shot];
    const float wsrc = a.src_scale * a.wav[(a.wav_per_shot ? (long long)shot * g.nt : 0) + a.n];
    for (int i = tid; i < TZ * TX; i += NTH) {
        int r = i / TX, c = i - r * TX;
        int z = tz0 + r, x = tx0 + c;
        if (z >= g.Nz || x >= g.Nx) continue;
        long long cell = (long long)z * pitch + x;
        const float *vxr = sVx + r * VXW + c + M;
        const float *vzc = sVz + (r + M) * TX + c;
        float qx = 0.f, qz = 0.f;
#pragma unroll
        for (int l = 1; l <= M; ++l) {
            qx += g.cx[l - 1] * (vxr[l - 1] - vxr[-l]);
            qz += g.cz[l - 1] * (vzc[(l - 1) * TX] - vzc[-l * TX]);
        }
        bool pmlx = (x <= x0 - 1) || (x >= x1);
        bool pmlz = (z <= z0 - 1) || (z >= z1);
        float dqx = 0.f, dqz = 0.f;
        if (BORN) {
            const float *dvxr = vxr + TZ * VXW;
            const float *dvzc = vzc + G::VZH * TX;
#pragma unroll
            for (int l = 1; l <= M; ++l) {
                dqx += g.cx[l - 1] * (dvxr[l - 1] - dvxr[-l]);
                dqz += g.cz[l - 1] * (dvzc[(l - 1) * TX] - dvzc[-l * TX]);
            }
        }
        if (pmlx) {
            float ps = a.pml.bi[2][x] * psiv[0 * plane + cell] + a.pml.ai[2][x] * qx;
            psiv[0 * plane + cell] = ps;
            qx += ps;
            if (BORN) {
                float ds = a.pml.bi[2][x] * psiv[2 * plane + cell] + a.pml.ai[2][x] * dqx;
                psiv[2 * plane + cell] = ds;
                dqx += ds;
            }
        }
        if (pmlz) {
            float ps = a.pml.bi[0][z] * psiv[1 * plane + cell] + a.pml.ai[0][z] * qz;
            psiv[1 * plane + cell] = ps;
            qz += ps;
            if (BORN) {
                float ds = a.pml.bi[0][z] * psiv[3 * plane + cell] + a.pml.ai[0][z] * dqz;
                psiv[3 * plane + cell] = ds;
                dqz += ds;
            }
        }
        float Q = qx + qz;
        float kd = __ldg(a.kdt + cell);
        float p0 = sP[(r + H) * SX + c + HX];
        float pn = p0 - kd * Q;
        if (cell == src) pn += wsrc;
        out[F_P * plane + cell] = pn;
        if (BORN) {
            float dp0 = sP[SZ * SX + (r + H) * SX + c + HX];
            out[(F_D + F_P) * plane + cell] = dp0 - kd * (dqx + dqz) - __ldg(a.dkdt + cell) * Q;
        }
        if (BANDS) {
            long long b = pband_index(z - z0, x - x0, M, g.nz, g.nx);
            if (b >= 0) band_put(a.bands, a.bands.p, bandoff + b, p0);
        }
        if (HESS) {
            int iz = z - z0, ix = x - x0;
            if (iz >= 0 && iz < g.nz && ix >= 0 && ix < g.nx) {
                float bi = __ldg(a.binv + cell);
                float hr = 0.5f * (sHx[r * (TX + 1) + c + 1] + sHx[r * (TX + 1) + c] +
                                   sHz[(r + 1) * TX + c] + sHz[r * TX + c]) / (bi * bi);
                float kq = kd * Q / dt;
                a.hess[slot * plane + cell] += dt * (hr + kq * kq);
            }
        }
    }

    if (BORN) {
        // record dp^{n+1} at the receivers of this tile
        __syncthreads();
        int t = shot * a.trec.ntiles + blockIdx.y * gridDim.x + blockIdx.x;
        int b = a.trec.ptr[t], e = a.trec.ptr[t + 1];
        for (int i = b + tid; i < e; i += NTH) {
            int2 rc = a.trec.rec[i];
            a.dstage[(long long)rc.y * g.nt + a.n] = out[(F_D + F_P) * plane + rc.x];
        }
    }
}

// ---------------------------------------------------------------------------
// Reverse step n (n = nt-1 .. 0) of L^T. Input state: background p^n,
// v^{n+1/2}; adjoint lambda_p (with the residual of step n already added),
// lambda_v, CPML memories. The step applies the transposed Born sub-steps
// S4^T, S3^T, S2^T, S1^T, accumulates the two zero-lag images (Eqs. gradkappa,
// gradrho in their discrete transposed form), reconstructs p^{n-1}, v^{n-1/2}
// in the interior from the saved boundary bands, and pre-adds the residual of
// step n-1 to the new lambda_p.
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(NTH) k_adj2d(const Step2D a)
{
    using G = Geo<M>;
    constexpr int H = G::H, HX = G::HX, SX = G::SX, SZ = G::SZ, VXW = G::VXW, VZH = G::VZH;
    constexpr int SX4 = SX / 4;
    extern __shared__ __align__(16) float smem[];
    float *sP = smem;                 // [SZ][SX] background p^n
    float *sUx = sP + SZ * SX;        // [SZ][SX] kdt*lp - ai_x*(lpsi_vx - kdt*lp)
    float *sUz = sUx + SZ * SX;       // [SZ][SX] same along z
    float *sVxo = sUz + SZ * SX;      // [TZ][VXW] background vx^{n+1/2}
    float *sVxn = sVxo + TZ * VXW;    // [TZ][VXW] background vx^{n-1/2}
    float *sWx = sVxn + TZ * VXW;     // [TZ][VXW] dt*bu*lvx - ah*lpsi_px
    float *sVzo = sWx + TZ * VXW;     // [VZH][TX]
    float *sVzn = sVzo + VZH * TX;
    float *sWz = sVzn + VZH * TX;
    float *sPix = sWz + VZH * TX;     // [TZ][TX+1]  Gx*lvx at half nodes tx0-1 .. tx0+TX-1
    float *sPiz = sPix + TZ * (TX + 1);  // [TZ+1][TX]

    const GridDev &g = a.g;
    const int tid = threadIdx.x;
    const int tx0 = blockIdx.x * TX, tz0 = blockIdx.y * TZ;
    const int slot = blockIdx.z, shot = a.shot0 + slot;
    const int pitch = g.pitch;
    const long long plane = g.plane;
    const float *in = a.in + slot * a.sstride;
    float *out = a.out + slot * a.sstride;
    const float dt = g.dt;
    const int n = a.n;
    const int x0 = g.x0, x1 = g.x0 + g.nx, z0 = g.z0, z1 = g.z0 + g.nz;
    const bool recon = n > 0;
    const long long bandprev = ((long long)shot * g.nt + (n - 1)) * a.bands.nb;

    load_box<M>(sP, in + A_P * plane, g, tz0, tx0);
    for (int i = tid; i < SZ * SX4; i += NTH) {
        int rz = i / SX4, q = i - rz * SX4;
        int z = tz0 - H + rz, xq = tx0 - HX + 4 * q;
        float lp[4] = {0.f, 0.f, 0.f, 0.f}, kd[4] = {0.f, 0.f, 0.f, 0.f};
        bool ok = z >= 0 && z < g.Nz && xq >= 0 && xq < g.pitch;
        if (ok) {
            long long cell = (long long)z * pitch + xq;
            float4 l4 = __ldg(reinterpret_cast<const float4 *>(in + A_LP * plane + cell));
            float4 k4 = __ldg(reinterpret_cast<const float4 *>(a.kdt + cell));
            lp[0] = l4.x; lp[1] = l4.y; lp[2] = l4.z; lp[3] = l4.w;
            kd[0] = k4.x; kd[1] = k4.y; kd[2] = k4.z; kd[3] = k4.w;
        }
        bool pmlz = ok && ((z <= z0 - 1) || (z >= z1));
        float ux[4], uz[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float l1 = kd[e] * lp[e];
            ux[e] = l1;
            uz[e] = l1;
            int x = xq + e;
            if (ok && x < g.Nx) {
                long long cell = (long long)z * pitch + x;
                if ((x <= x0 - 1) || (x >= x1))
                    ux[e] = l1 - a.pml.ai[2][x] * (__ldg(in + A_LPVX * plane + cell) - l1);
                if (pmlz)
                    uz[e] = l1 - a.pml.ai[0][z] * (__ldg(in + A_LPVZ * plane + cell) - l1);
            }
        }
        *reinterpret_cast<float4 *>(sUx + rz * SX + 4 * q) = make_float4(ux[0], ux[1], ux[2], ux[3]);
        *reinterpret_cast<float4 *>(sUz + rz * SX + 4 * q) = make_float4(uz[0], uz[1], uz[2], uz[3]);
    }
    for (int i = tid; i < G::NVX; i += NTH) {
        int r = i / (VXW - 1), ci = i - r * (VXW - 1);
        int z = tz0 + r, j = tx0 - M + ci;
        sVxo[r * VXW + ci] = (z < g.Nz && j >= 0 && j < g.Nx)
                                 ? __ldg(in + A_VX * plane + (long long)z * pitch + j) : 0.f;
    }
    for (int i = tid; i < G::NVZ; i += NTH) {
        int r = i / TX, c = i - r * TX;
        int k = tz0 - M + r, x = tx0 + c;
        sVzo[r * TX + c] = (k >= 0 && k < g.Nz && x < g.Nx)
                               ? __ldg(in + A_VZ * plane + (long long)k * pitch + x) : 0.f;
    }
    __syncthreads();

    // ---- half-node stage along x: lambda_vx (S4^T, S3^T), lambda_psi_px,
    //      background vx^{n-1/2}, rho-image products
    for (int i = tid; i < G::NVX; i += NTH) {
        int r = i / (VXW - 1), ci = i - r * (VXW - 1);
        int z = tz0 + r, j = tx0 - M + ci;
        float w = 0.f, vn = 0.f, pi = 0.f;
        if (z < g.Nz && j >= 0 && j < g.Nx) {
            long long cell = (long long)z * pitch + j;
            bool own = ci >= M && ci < M + TX;
            const float *ur = sUx + (r + H) * SX + (ci - M + HX);
            const float *pr = sP + (r + H) * SX + (ci - M + HX);
            float du = 0.f, Gx = 0.f;
#pragma unroll
            for (int l = 1; l <= M; ++l) {
                du += g.cx[l - 1] * (ur[l] - ur[1 - l]);
                Gx += g.cx[l - 1] * (pr[l] - pr[1 - l]);
            }
            float lv = __ldg(in + A_LVX * plane + cell) + du;
            float bu = 0.5f * (__ldg(a.binv + cell) + __ldg(a.binv + (j + 1 < g.Nx ? cell + 1 : cell)));
            float dtbu = dt * bu;
            w = dtbu * lv;
            if ((j <= x0 - 2) || (j >= x1)) {
                float l1 = __ldg(in + A_LPPX * plane + cell) - dtbu * lv;
                w -= a.pml.ah[2][j] * l1;
                if (own) out[A_LPPX * plane + cell] = a.pml.bh[2][j] * l1;
            }
            if (own) out[A_LVX * plane + cell] = lv;
            pi = Gx * lv;
            if (recon) {
                int iz = z - z0, ix = j - x0;
                if (iz >= 0 && iz < g.nz) {
                    if (ix >= 0 && ix < g.nx) vn = sVxo[r * VXW + ci] + dtbu * Gx;
                    else if ((ix >= -M && ix < 0) || (ix >= g.nx && ix < g.nx + M))
                        vn = band_get(a.bands, a.bands.v, bandprev + band_xstrip(iz, ix, M, g.nz, g.nx));
                }
                if (own) out[A_VX * plane + cell] = vn;
            }
        }
        sWx[r * VXW + ci] = w;
        sVxn[r * VXW + ci] = vn;
        if (ci >= M - 1 && ci < M + TX) sPix[r * (TX + 1) + (ci - M + 1)] = pi;
    }
    // ---- half-node stage along z
    for (int i = tid; i < G::NVZ; i += NTH) {
        int r = i / TX, c = i - r * TX;
        int k = tz0 - M + r, x = tx0 + c;
        float w = 0.f, vn = 0.f, pi = 0.f;
        if (k >= 0 && k < g.Nz && x < g.Nx) {
            long long cell = (long long)k * pitch + x;
            bool own = r >= M && r < M + TZ;
            const float *uc = sUz + (r - M + H) * SX + (c + HX);
            const float *pc = sP + (r - M + H) * SX + (c + HX);
            float du = 0.f, Gz = 0.f;
#pragma unroll
            for (int l = 1; l <= M; ++l) {
                du += g.cz[l - 1] * (uc[l * SX] - uc[(1 - l) * SX]);
                Gz += g.cz[l - 1] * (pc[l * SX] - pc[(1 - l) * SX]);
            }
            float lv = __ldg(in + A_LVZ * plane + cell) + du;
            float bu = 0.5f * (__ldg(a.binv + cell) + __ldg(a.binv + (k + 1 < g.Nz ? cell + pitch : cell)));
            float dtbu = dt * bu;
            w = dtbu * lv;
            if ((k <= z0 - 2) || (k >= z1)) {
                float l1 = __ldg(in + A_LPPZ * plane + cell) - dtbu * lv;
                w -= a.pml.ah[0][k] * l1;
                if (own) out[A_LPPZ * plane + cell] = a.pml.bh[0][k] * l1;
            }
            if (own) out[A_LVZ * plane + cell] = lv;
            pi = Gz * lv;
            if (recon) {
                int iz = k - z0, ix = x - x0;
                if (ix >= 0 && ix < g.nx) {
                    if (iz >= 0 && iz < g.nz) vn = sVzo[r * TX + c] + dtbu * Gz;
                    else if ((iz >= -M && iz < 0) || (iz >= g.nz && iz < g.nz + M))
                        vn = band_get(a.bands, a.bands.v, bandprev + band_zstrip(iz, ix, M, g.nz, g.nx));
                }
                if (own) out[A_VZ * plane + cell] = vn;
            }
        }
        sWz[r * TX + c] = w;
        sVzn[r * TX + c] = vn;
        if (r >= M - 1 && r < M + TZ) sPiz[(r - M + 1) * TX + c] = pi;
    }
    __syncthreads();

    // ---- node stage on the own tile
    const int src = a.src_cell[shot];
    const float wsrc = recon ? a.src_scale * a.wav[(a.wav_per_shot ? (long long)shot * g.nt : 0) + n - 1]
                             : 0.f;
    float2 *img = a.img + slot * plane;
    for (int i = tid; i < TZ * TX; i += NTH) {
        int r = i / TX, c = i - r * TX;
        int z = tz0 + r, x = tx0 + c;
        if (z >= g.Nz || x >= g.Nx) continue;
        long long cell = (long long)z * pitch + x;
        const float *vxo = sVxo + r * VXW + c + M;
        const float *vzo = sVzo + (r + M) * TX + c;
        const float *wxr = sWx + r * VXW + c + M;
        const float *wzc = sWz + (r + M) * TX + c;
        float Q = 0.f, dw = 0.f;
#pragma unroll
        for (int l = 1; l <= M; ++l) {
            Q += g.cx[l - 1] * (vxo[l - 1] - vxo[-l]) + g.cz[l - 1] * (vzo[(l - 1) * TX] - vzo[-l * TX]);
            dw += g.cx[l - 1] * (wxr[l - 1] - wxr[-l]) + g.cz[l - 1] * (wzc[(l - 1) * TX] - wzc[-l * TX]);
        }
        float lp1 = __ldg(in + A_LP * plane + cell);
        float kd = __ldg(a.kdt + cell);
        int iz = z - z0, ix = x - x0;
        bool inner = iz >= 0 && iz < g.nz && ix >= 0 && ix < g.nx;
        if (inner) {
            float2 acc = img[cell];
            acc.x += Q * lp1;
            acc.y += (sPix[r * (TX + 1) + c + 1] + sPix[r * (TX + 1) + c]) +
                     (sPiz[(r + 1) * TX + c] + sPiz[r * TX + c]);
            img[cell] = acc;
        }
        out[A_LP * plane + cell] = lp1 + dw;
        if ((x <= x0 - 1) || (x >= x1))
            out[A_LPVX * plane + cell] = a.pml.bi[2][x] * (__ldg(in + A_LPVX * plane + cell) - kd * lp1);
        if ((z <= z0 - 1) || (z >= z1))
            out[A_LPVZ * plane + cell] = a.pml.bi[0][z] * (__ldg(in + A_LPVZ * plane + cell) - kd * lp1);
        if (recon) {
            float pn = 0.f;
            if (inner) {
                const float *vxn = sVxn + r * VXW + c + M;
                const float *vzn = sVzn + (r + M) * TX + c;
                float qn = 0.f;
#pragma unroll
                for (int l = 1; l <= M; ++l)
                    qn += g.cx[l - 1] * (vxn[l - 1] - vxn[-l]) + g.cz[l - 1] * (vzn[(l - 1) * TX] - vzn[-l * TX]);
                pn = sP[(r + H) * SX + c + HX] + kd * qn;
                if (cell == src) pn -= wsrc;
            } else {
                long long b = pband_index(iz, ix, M, g.nz, g.nx);
                if (b >= 0) pn = band_get(a.bands, a.bands.p, bandprev + b);
            }
            out[A_P * plane + cell] = pn;
        }
    }

    if (recon) {
        // pre-add the residual of step n-1 at the receivers of this tile
        __syncthreads();
        int t = shot * a.trec.ntiles + blockIdx.y * gridDim.x + blockIdx.x;
        int b = a.trec.ptr[t], e = a.trec.ptr[t + 1];
        for (int i = b + tid; i < e; i += NTH) {
            int2 rc = a.trec.rec[i];
            if (i > b && a.trec.rec[i - 1].x == rc.x) continue;  // run handled by its first entry
            float add = 0.f;
            for (int k = i; k < e && a.trec.rec[k].x == rc.x; ++k)
                add += a.dstage[(long long)a.trec.rec[k].y * g.nt + (n - 1)];
            out[A_LP * plane + rc.x] += add;
        }
    }
}

template <int M>
size_t fwd_smem_M(bool born, bool hess)
{
    using G = Geo<M>;
    int nf = born ? 2 : 1;
    size_t f = (size_t)nf * (G::SZ * G::SX + TZ * G::VXW + G::VZH * TX);
    if (hess) f += TZ * (TX + 1) + (TZ + 1) * TX;
    return f * sizeof(float);
}

template <int M>
size_t adj_smem_M()
{
    using G = Geo<M>;
    size_t f = 3 * (size_t)G::SZ * G::SX + 3 * (size_t)TZ * G::VXW + 3 * (size_t)G::VZH * TX +
               TZ * (TX + 1) + (TZ + 1) * TX;
    return f * sizeof(float);
}

template <int M, bool BORN, bool BANDS, bool HESS>
cudaError_t set_fwd_attr()
{
    return cudaFuncSetAttribute(k_fwd2d<M, BORN, BANDS, HESS>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fwd_smem_M<M>(BORN, HESS));
}

template <int M>
cudaError_t configure_M()
{
    cudaError_t e;
    if ((e = set_fwd_attr<M, true, false, false>()) != cudaSuccess) return e;
    if ((e = set_fwd_attr<M, false, true, false>()) != cudaSuccess) return e;
    if ((e = set_fwd_attr<M, false, true, true>()) != cudaSuccess) return e;
    if ((e = set_fwd_attr<M, false, false, false>()) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_adj2d<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)adj_smem_M<M>());
}

template <int M>
cudaError_t launch_fwd_M(const Step2D &a, int batch, bool born, bool bands, bool hess,
                         cudaStream_t s)
{
    dim3 grid((a.g.Nx + TX - 1) / TX, (a.g.Nz + TZ - 1) / TZ, batch);
    size_t sm = fwd_smem_M<M>(born, hess);
    if (born) k_fwd2d<M, true, false, false><<<grid, NTH, sm, s>>>(a);
    else if (bands && hess) k_fwd2d<M, false, true, true><<<grid, NTH, sm, s>>>(a);
    else if (bands) k_fwd2d<M, false, true, false><<<grid, NTH, sm, s>>>(a);
    else k_fwd2d<M, false, false, false><<<grid, NTH, sm, s>>>(a);
    return cudaGetLastError();
}

template <int M>
cudaError_t launch_adj_M(const Step2D &a, int batch, cudaStream_t s)
{
    dim3 grid((a.g.Nx + TX - 1) / TX, (a.g.Nz + TZ - 1) / TZ, batch);
    k_adj2d<M><<<grid, NTH, adj_smem_M<M>(), s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t fwd2d_smem(int M, bool born, bool hess)
{
    return M == 2 ? fwd_smem_M<2>(born, hess) : fwd_smem_M<4>(born, hess);
}

size_t adj2d_smem(int M) { return M == 2 ? adj_smem_M<2>() : adj_smem_M<4>(); }

cudaError_t configure_2d_kernels()
{
    cudaError_t e = configure_M<2>();
    if (e != cudaSuccess) return e;
    return configure_M<4>();
}

cudaError_t launch_fwd2d(const Step2D &a, int batch, bool born, bool save_bands, bool hess,
                         cudaStream_t s)
{
    if (a.g.M == 2) return launch_fwd_M<2>(a, batch, born, save_bands, hess, s);
    return launch_fwd_M<4>(a, batch, born, save_bands, hess, s);
}

cudaError_t launch_adj2d(const Step2D &a, int batch, cudaStream_t s)
{
    if (a.g.M == 2) return launch_adj_M<2>(a, batch, s);
    return launch_adj_M<4>(a, batch, s);
}

}  // namespace lsrtm
