// Fused 3D time-step kernels: one launch advances every shot of a batch by
// one time step of the Born operator (Eq. scattereqln driven by Eq. 1) or of
// its exact transpose (App. A), reading each state field once from HBM and
// writing it once (ping-pong buffers).
//
// A CTA of 384 threads owns a 32 x 12 tile of (x, y) columns, one column per
// thread, and marches down a z-chunk (two CTAs per SM):
//   * z stencils: per-thread register rings of length 2M (+1 look-ahead),
//     shifted after every row;
//   * x and y stencils: shared-memory tiles of the current row. Every tile a
//     row needs (the centre column block, the x-extended and y-extended
//     halo blocks, the model) arrives by TMA (cp.async.bulk.tensor, one
//     elected thread) into a 2-deep stage ring guarded by mbarriers, one
//     row ahead of the compute; the tensor maps zero-fill outside the padded
//     array, which is the operators' boundary convention;
//   * the velocity (half-node) stage is recomputed on the x and y halos, so
//     the pressure stage of the same row needs nothing from other CTAs and a
//     step needs no grid-wide barrier.
// A background field and its partner (scattered or adjoint) are float2
// pairs, so one 8-byte access and one packed FFMA2 serve both.
//
// Every mbarrier wait is bounded: after kWaitLimit polls the CTA sets the
// error word, waits (bounded) for its copies in flight and returns; the host
// reports the error.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "lsrtm_internal.cuh"
#include "tma.cuh"

namespace lsrtm {
namespace {

constexpr int TX = kTile3X, TY = kTile3Y, NTH = TX * TY;
constexpr int PD = 2;                       // stage ring depth
constexpr int kMinBlocks = 2;               // resident CTAs per SM the register budget targets

// ---- packed arithmetic
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float a, float2 b, float2 c) { return __ffma2_rn(f2(a), b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float a, float2 b) { return __fmul2_rn(f2(a), b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(f2(-1.f), b, a); }

// sum_l c_l (fa(l) - fb(l)), l = 1..M: M independent differences, then one
// multiply-add chain of depth M.
template <int M, class FA, class FB>
__device__ __forceinline__ float2 st2(const float *c, FA fa, FB fb)
{
    float2 d[M];
#pragma unroll
    for (int l = 0; l < M; ++l) d[l] = sub2(fa(l + 1), fb(l + 1));
    float2 acc = mul2(c[0], d[0]);
#pragma unroll
    for (int l = 1; l < M; ++l) acc = fma2(c[l], d[l], acc);
    return acc;
}
template <int M, class FA, class FB>
__device__ __forceinline__ float st1(const float *c, FA fa, FB fb)
{
    float d[M];
#pragma unroll
    for (int l = 0; l < M; ++l) d[l] = fa(l + 1) - fb(l + 1);
    float acc = c[0] * d[0];
#pragma unroll
    for (int l = 1; l < M; ++l) acc = fmaf(c[l], d[l], acc);
    return acc;
}

// Free surface (method of images about row z0): ghost node rows r < z0 read
// their mirror row with the sign flipped (p odd), ghost half rows k < z0 their
// mirror half row (v_z even).
__device__ __forceinline__ int node_src_row(const GridDev &g, int r) { return (g.fs && r < g.z0) ? fs_node_row(g, r) : r; }
__device__ __forceinline__ int half_src_row(const GridDev &g, int k) { return (g.fs && k < g.z0) ? fs_half_row(g, k) : k; }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// ---- shared memory, mbarriers and TMA (tma.cuh)
using tma::al128;
using tma::kWaitLimit;
using tma::mbar_expect;
using tma::mbar_init;
using tma::mbar_wait;
using tma::su32;
__device__ __forceinline__ void tma4(void *dst, const CUtensorMap &m, int x, int y, int z, int q, uint64_t *b)
{
    tma::load4(dst, m, x, y, z, q, b);
}

// Tile geometry for half-width M. Box shapes (x extent in elements, rows):
//   core  TX x TY                      the thread block's own columns
//   xbox  XW1 x TY   from x0 - 4       half nodes [x0-M, x0+TX+M-2] and their rho pairs
//   ybox  TX x YH1   from y0 - M       half nodes [y0-M, y0+TY+M-2]
//   ybr   XW1 x YHB  from (x0-4, y0-M) rho pairs of both half-node directions
//   wide  XW2 x YH2  from (x0-XO2, y0-YO2) nodes feeding the halo stencils
// Every x start is a multiple of 4 elements, so each TMA copy starts on a
// 16-byte boundary for float and float2 elements alike.
template <int M>
struct Geo {
    static constexpr int W = 2 * M;
    static constexpr int XO1 = 4, XW1 = TX + 8;
    static constexpr int XO2 = (2 * M + 3) / 4 * 4, XW2 = TX + 2 * XO2;
    static constexpr int YO1 = M, YH1 = TY + 2 * M - 1, YHB = TY + 2 * M;
    static constexpr int YO2 = 2 * M - 1, YH2 = TY + 4 * M - 2;
    static constexpr int NXI = TX + 2 * M - 1;   // half nodes per row of the x halo stage
    static_assert(XO1 >= M && XO2 >= 2 * M - 1, "halo offsets");
};

// ---------------------------------------------------------------------------
// Born modelling step n -> n+1.
// ---------------------------------------------------------------------------
template <int M>
struct BornSmem {
    using G = Geo<M>;
    // stage layout (bytes)
    static constexpr unsigned PA = 0;                                     // p, row z+W-1, core
    static constexpr unsigned VZ = PA + al128(TX * TY * 8);               // vz, half row z+M-1, core
    static constexpr unsigned BK = VZ + al128(TX * TY * 8);               // br pairs, row z+M, core
    static constexpr unsigned KD = BK + al128(TX * TY * 8);               // kd pairs, row z, core
    static constexpr unsigned PZ = KD + al128(TX * TY * 8);               // psi_pz, half row z+M-1, core
    static constexpr unsigned PW = PZ + al128(TX * TY * 8);               // p, row z, wide
    static constexpr unsigned VX = PW + al128(G::XW2 * G::YH2 * 8);       // vx, row z, xbox
    static constexpr unsigned VY = VX + al128(G::XW1 * TY * 8);           // vy, row z, ybox
    static constexpr unsigned BR = VY + al128(TX * G::YH1 * 8);           // br pairs, row z, ybr
    static constexpr unsigned PX = BR + al128(G::XW1 * G::YHB * 8);       // psi_px, row z, xbox
    static constexpr unsigned PY = PX + al128(G::XW1 * TY * 8);           // psi_py, row z, ybox
    static constexpr unsigned STAGE = PY + al128(TX * G::YH1 * 8);
    // after the stages: the new vx / vy of the row (half-node halos)
    static constexpr unsigned OVX = PD * STAGE;
    static constexpr unsigned OVY = OVX + al128(G::XW1 * TY * 8);
    static constexpr unsigned BAR = OVY + al128(TX * G::YH1 * 8);
    static constexpr unsigned TOTAL = BAR + 64 + 128;   // + alignment slack
};

}  // namespace

size_t fused3d_born_smem(int M) { return M == 2 ? BornSmem<2>::TOTAL : BornSmem<4>::TOTAL; }

namespace {

template <int M>
__device__ __forceinline__ void born_issue(const Step3F &a, unsigned char *st, uint64_t *bar, int slot, int x0,
                                           int y0, int z, int zc0, bool px, bool py)
{
    using G = Geo<M>;
    using S = BornSmem<M>;
    const GridDev &g = a.g;
    const int k = z + M - 1, r = z + G::W - 1;
    const bool main = z >= zc0;
    const bool pzs = k >= 0 && k < g.Nz && (k <= g.z0 - 2 || k >= g.z0 + g.nz);
    const int q = slot * a.in_pairs;   // pair-plane index of the slot's first field
    unsigned bytes = 3 * TX * TY * 8 + (pzs ? TX * TY * 8 : 0);
    if (main) {
        bytes += TX * TY * 8 + G::XW2 * G::YH2 * 8 + G::XW1 * TY * 8 + TX * G::YH1 * 8 + G::XW1 * G::YHB * 8;
        if (px) bytes += G::XW1 * TY * 8;
        if (py) bytes += TX * G::YH1 * 8;
    }
    // x coordinates in floats (pairs x 2); each a multiple of 4 (16 bytes)
    const int xc = 2 * x0, x1 = 2 * (x0 - G::XO1), x2 = 2 * (x0 - G::XO2);
    if ((xc | x1 | x2) & 3) {   // never issue a misaligned copy
        atomicOr(a.err, 2);
        return;
    }
    mbar_expect(bar, bytes);
    tma4(st + S::PA, a.in_core, xc, y0, node_src_row(g, r), q + F3_P, bar);
    tma4(st + S::VZ, a.in_core, xc, y0, half_src_row(g, k), q + F3_VZ, bar);
    tma4(st + S::BK, a.m_core, xc, y0, k + 1, 1, bar);
    if (pzs) tma4(st + S::PZ, a.in_core, xc, y0, k, q + F3_PPZ, bar);
    if (main) {
        tma4(st + S::KD, a.m_core, xc, y0, z, 0, bar);
        tma4(st + S::PW, a.in_wide, x2, y0 - G::YO2, z, q + F3_P, bar);
        tma4(st + S::VX, a.in_xbox, x1, y0, z, q + F3_VX, bar);
        tma4(st + S::VY, a.in_ybox, xc, y0 - G::YO1, z, q + F3_VY, bar);
        tma4(st + S::BR, a.m_ybr, x1, y0 - G::YO1, z, 1, bar);
        if (px) tma4(st + S::PX, a.in_xbox, x1, y0, z, q + F3_PPX, bar);
        if (py) tma4(st + S::PY, a.in_ybox, xc, y0 - G::YO1, z, q + F3_PPY, bar);
    }
}

template <int M>
__global__ void __launch_bounds__(NTH, kMinBlocks) k3f_born(const __grid_constant__ Step3F a)
{
    if (guard_tripped(a.g)) return;
    using G = Geo<M>;
    using S = BornSmem<M>;
    constexpr int W = G::W;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((128u - (su32(smem_raw) & 127u)) & 127u);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + S::BAR);
    float2 *oVX = reinterpret_cast<float2 *>(sm + S::OVX);
    float2 *oVY = reinterpret_cast<float2 *>(sm + S::OVY);

    const GridDev &g = a.g;
    const int t = threadIdx.x, tx = t % TX, ty = t / TX;
    const int nzc = (g.Nz + a.tzc - 1) / a.tzc;
    const int slot = blockIdx.z / nzc, zcn = blockIdx.z - slot * nzc;
    const int shot = a.shot0 + slot;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool colok = x < g.Nx && y < g.Ny;
    const int zc0 = zcn * a.tzc, zc1 = min(zc0 + a.tzc, g.Nz);
    const int zstart = zc0 - W;
    const float dt = g.dt;
    const long long plane = g.plane;
    const long long cxy = (long long)y * g.pitch + x;
    // CTA-uniform: does the tile's x (y) halo reach a CPML strip?
    const bool px = (x0 - M <= g.x0 - 2) || (x0 + TX + M - 2 >= g.x0 + g.nx);
    const bool py = (y0 - M <= g.y0 - 2) || (y0 + TY + M - 2 >= g.y0 + g.ny);
    float2 *out = reinterpret_cast<float2 *>(a.out) + slot * a.out_pairs * plane;
    float2 *psv = reinterpret_cast<float2 *>(a.psiv) + slot * a.psiv_pairs * plane;   // in place: x y z
    const int src = a.src_cell[shot];
    const float wsrc = a.src_scale * a.wav[(a.wav_per_shot ? (long long)shot * g.nt : 0) + a.n];

    if (t == 0) {
        for (int i = 0; i < PD; ++i) mbar_init(bar + i);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (t == 0) {
        for (int j = 0; j < PD - 1; ++j)
            if (zstart + j < zc1) born_issue<M>(a, sm + j * S::STAGE, bar + j, slot, x0, y0, zstart + j, zc0, px, py);
    }

    // z rings: P[m] = p^n at row z + m (m = 0..W-1, P[W-1] filled each row),
    // VZ[m] = vz^{n+1/2} at half row z + m - M.
    float2 P[W], VZ[W];
    {
        const float2 *pin = reinterpret_cast<const float2 *>(a.in) + slot * a.in_pairs * plane + F3_P * plane;
#pragma unroll
        for (int m = 0; m < W - 1; ++m) {
            const int zr = zstart + m, zs = node_src_row(g, zr);
            const float2 v = (colok && zs >= 0 && zs < g.Nz) ? pin[zs * g.rowz + cxy] : make_float2(0.f, 0.f);
            P[m] = zs != zr ? neg2(v) : v;
        }
#pragma unroll
        for (int m = 0; m < W; ++m) VZ[m] = make_float2(0.f, 0.f);
    }
    float2 br_old = make_float2(0.f, 0.f);
    {
        const int kk = zstart + M - 1;
        if (colok && kk >= 0 && kk < g.Nz) br_old = a.br2[kk * g.rowz + cxy];
    }

    bool failed = false;
    int fail_row = 0;
    const int pl = (int)plane;   // in-slot offsets fit in 32 bits (checked by the host)
    const int rowz = (int)g.rowz, pitch = g.pitch;
    const int cxy32 = y * pitch + x;
    for (int z = zstart; z < zc1; ++z) {
        const int j = z - zstart;
        const bool to = !mbar_wait(bar + j % PD, (unsigned)(j / PD) & 1u);
        // (this barrier also certifies that every thread is done with row z-1,
        // its stage and the vx / vy tiles)
        if (__syncthreads_or(to)) {
            failed = true;
            fail_row = z;
            break;
        }
        // the last warp has no item in the last round of the halo loop: it
        // refills the stage of row z-1 with row z+PD-1
        if (t == NTH - 1 && z + PD - 1 < zc1) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            born_issue<M>(a, sm + ((j + PD - 1) % PD) * S::STAGE, bar + (j + PD - 1) % PD, slot, x0, y0, z + PD - 1,
                          zc0, px, py);
        }
        const unsigned char *st = sm + (j % PD) * S::STAGE;
        const float2 *cPA = reinterpret_cast<const float2 *>(st + S::PA);
        const float2 *cVZ = reinterpret_cast<const float2 *>(st + S::VZ);
        const float2 *cBK = reinterpret_cast<const float2 *>(st + S::BK);
        const float2 *cPZ = reinterpret_cast<const float2 *>(st + S::PZ);
        const int k = z + M - 1;

        // ---- vz at half row k (column-local)
        P[W - 1] = (g.fs && z + W - 1 < g.z0) ? neg2(cPA[t]) : cPA[t];   // ghost rows: -p(mirror)
        // (the last half row replicates the last node row's buoyancy)
        const float2 brk1 = k + 1 < g.Nz ? cBK[t] : make_float2(br_old.x, 0.f);
        float2 vzn = make_float2(0.f, 0.f);
        if (colok && k >= 0 && k < g.Nz) {
            float2 Gz = st2<M>(g.cz, [&](int l) { return P[M - 1 + l]; }, [&](int l) { return P[M - l]; });
            const bool own = k >= zc0 && k < zc1;
            if (k <= g.z0 - 2 || k >= g.z0 + g.nz) {
                const float2 ps = fma2(a.pml.bh[0][k], cPZ[t], mul2(a.pml.ah[0][k], Gz));
                if (own) out[F3_PPZ * pl + k * rowz + cxy32] = ps;
                Gz = add2(Gz, ps);
            }
            const float bu = 0.5f * (br_old.x + brk1.x);
            vzn = fma2(-dt * bu, Gz, cVZ[t]);
            vzn.y = fmaf(0.5f * dt * (br_old.y + brk1.y), Gz.x, vzn.y);
            if (own) out[F3_VZ * pl + k * rowz + cxy32] = vzn;
        }
        br_old = brk1;
        VZ[W - 1] = vzn;

        if (z >= zc0) {
            const float2 *cKD = reinterpret_cast<const float2 *>(st + S::KD);
            const float2 *wP = reinterpret_cast<const float2 *>(st + S::PW);
            const float2 *bVX = reinterpret_cast<const float2 *>(st + S::VX);
            const float2 *bVY = reinterpret_cast<const float2 *>(st + S::VY);
            const float2 *bBR = reinterpret_cast<const float2 *>(st + S::BR);
            const float2 *bPX = reinterpret_cast<const float2 *>(st + S::PX);
            const float2 *bPY = reinterpret_cast<const float2 *>(st + S::PY);
            const int rz = z * rowz;
            // ---- velocities on the halos of the row, one loop over both:
            // items [0, NVX) are vx at half nodes xh = x0 - M + jx of row iy,
            // the rest vy at half nodes yh = y0 - M + jy of column ix
            constexpr int NVX = TY * G::NXI, NIT = NVX + G::YH1 * TX;
            for (int i = t; i < NIT; i += NTH) {
                if (i < NVX) {
                    const int iy = i / G::NXI, jx = i - iy * G::NXI;
                    const int xh = x0 - M + jx, yy = y0 + iy;
                    float2 v = make_float2(0.f, 0.f);
                    if (xh >= 0 && xh < g.Nx && yy < g.Ny) {
                        const float2 *pr = wP + (iy + G::YO2) * G::XW2 + (jx - M + G::XO2);
                        float2 Gx = st2<M>(g.cx, [&](int l) { return pr[l]; }, [&](int l) { return pr[1 - l]; });
                        const int cb = iy * G::XW1 + jx - M + G::XO1;   // xbox entry of half node xh
                        const bool own = jx >= M && jx < M + TX;
                        const int o = rz + yy * pitch + xh;
                        if (px && (xh <= g.x0 - 2 || xh >= g.x0 + g.nx)) {
                            const float2 ps = fma2(a.pml.bh[2][xh], bPX[cb], mul2(a.pml.ah[2][xh], Gx));
                            if (own) out[F3_PPX * pl + o] = ps;
                            Gx = add2(Gx, ps);
                        }
                        const float2 *brr = bBR + M * G::XW1 + cb;
                        const float2 b0 = brr[0];
                        const float2 b1 = xh + 1 >= g.Nx ? make_float2(b0.x, 0.f) : brr[1];
                        v = fma2(-dt * 0.5f * (b0.x + b1.x), Gx, bVX[cb]);
                        v.y = fmaf(0.5f * dt * (b0.y + b1.y), Gx.x, v.y);
                        if (own) out[F3_VX * pl + o] = v;
                    }
                    oVX[iy * G::XW1 + jx] = v;
                } else {
                    const int i2 = i - NVX;
                    const int jy = i2 / TX, ix = i2 - jy * TX;
                    const int yh = y0 - M + jy, xx = x0 + ix;
                    float2 v = make_float2(0.f, 0.f);
                    if (yh >= 0 && yh < g.Ny && xx < g.Nx) {
                        const float2 *pc = wP + (jy + M - 1) * G::XW2 + (ix + G::XO2);
                        float2 Gy = st2<M>(g.cy, [&](int l) { return pc[l * G::XW2]; },
                                           [&](int l) { return pc[(1 - l) * G::XW2]; });
                        const bool own = jy >= M && jy < M + TY;
                        const int o = rz + yh * pitch + xx;
                        if (py && (yh <= g.y0 - 2 || yh >= g.y0 + g.ny)) {
                            const float2 ps = fma2(a.pml.bh[1][yh], bPY[i2], mul2(a.pml.ah[1][yh], Gy));
                            if (own) out[F3_PPY * pl + o] = ps;
                            Gy = add2(Gy, ps);
                        }
                        const float2 *brc = bBR + jy * G::XW1 + ix + G::XO1;
                        const float2 b0 = brc[0];
                        const float2 b1 = yh + 1 >= g.Ny ? make_float2(b0.x, 0.f) : brc[G::XW1];
                        v = fma2(-dt * 0.5f * (b0.x + b1.x), Gy, bVY[i2]);
                        v.y = fmaf(0.5f * dt * (b0.y + b1.y), Gy.x, v.y);
                        if (own) out[F3_VY * pl + o] = v;
                    }
                    oVY[i2] = v;
                }
            }
            __syncthreads();
            // ---- pressure at row z on the thread's own column
            if (colok) {
                const float2 *vxr = oVX + ty * G::XW1 + tx + M;
                const float2 *vyc = oVY + (ty + M) * TX + tx;
                float2 Qx = st2<M>(g.cx, [&](int l) { return vxr[l - 1]; }, [&](int l) { return vxr[-l]; });
                float2 Qy = st2<M>(g.cy, [&](int l) { return vyc[(l - 1) * TX]; }, [&](int l) { return vyc[-l * TX]; });
                float2 Qz = st2<M>(g.cz, [&](int l) { return VZ[M + l - 1]; }, [&](int l) { return VZ[M - l]; });
                const int c = rz + cxy32;
                if (x <= g.x0 - 1 || x >= g.x0 + g.nx) {
                    float2 *m = psv + c;
                    const float2 ps = fma2(a.pml.bi[2][x], *m, mul2(a.pml.ai[2][x], Qx));
                    *m = ps;
                    Qx = add2(Qx, ps);
                }
                if (y <= g.y0 - 1 || y >= g.y0 + g.ny) {
                    float2 *m = psv + pl + c;
                    const float2 ps = fma2(a.pml.bi[1][y], *m, mul2(a.pml.ai[1][y], Qy));
                    *m = ps;
                    Qy = add2(Qy, ps);
                }
                if (z <= g.z0 - 1 || z >= g.z0 + g.nz) {
                    float2 *m = psv + 2 * pl + c;
                    const float2 ps = fma2(a.pml.bi[0][z], *m, mul2(a.pml.ai[0][z], Qz));
                    *m = ps;
                    Qz = add2(Qz, ps);
                }
                const float2 Q = add2(add2(Qx, Qy), Qz);
                const float2 kd = cKD[t];
                const float2 p0 = wP[(ty + G::YO2) * G::XW2 + tx + G::XO2];
                float2 pn = fma2(-kd.x, Q, p0);
                pn.y = fmaf(-kd.y, Q.x, pn.y);
                if (c == src) pn.x += wsrc;
                if (g.fs && z <= g.z0) pn = make_float2(0.f, 0.f);   // p = 0 on the free surface
                out[F3_P * pl + c] = pn;
            }
        }
#pragma unroll
        for (int m = 0; m < W - 1; ++m) {
            P[m] = P[m + 1];
            VZ[m] = VZ[m + 1];
        }
    }

    if (failed) {
        if (t == 0) {
            atomicOr(a.err, 1);
            // rows issued and not yet consumed: jf .. jf + PD - 1 (bounded waits)
            const int jf = fail_row - zstart;
            for (int jj = jf; jj < jf + PD && zstart + jj < zc1; ++jj)
                (void)mbar_wait(bar + jj % PD, (unsigned)(jj / PD) & 1u);
        }
        return;
    }
    // records dp^{n+1} at the receivers of this tile
    __syncthreads();
    const int ntile = (int)(gridDim.x * gridDim.y) * nzc;
    const int tile = shot * ntile + (zcn * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int b = a.trec.ptr[tile], e = a.trec.ptr[tile + 1];
    for (int i = b + t; i < e; i += NTH) {
        const int2 rc = a.trec.rec[i];
        a.dstage[(long long)rc.y * g.nt + a.n] = out[F3_P * plane + rc.x].y;   // (all rows written: barrier above)
    }
}

// ---------------------------------------------------------------------------
// Adjoint (migration) step n: the exact reverse-order transpose of the Born
// sub-steps, the zero-lag imaging condition and the reconstruction of the
// background p^{n-1}, v^{n-1/2} from p^n, v^{n+1/2} and the boundary bands
// (App. A), arranged as in the 2D kernel. State pairs (background, adjoint):
// (p, lambda_p) at nodes, (v_d, lambda_v_d) at half nodes; the lambda CPML
// memories as float planes. For the half-node stencils each node carries
// (p, u_d) with u_d = dt kappa lambda_p - a_d (lambda_psi_v_d - dt kappa
// lambda_p) (a_d nonzero only in the d strips).
// ---------------------------------------------------------------------------

// Face bands (as written by the 3D background kernels):
// [x faces 2M nz ny][y faces 2M nz nx][z faces 2M ny nx]; -1 if the interior
// offsets (iz, iy, ix) are not in the d face band.
__device__ __forceinline__ long long fband(const GridDev &g, int d, int iz, int iy, int ix)
{
    const int M = g.M;
    const int i = d == 0 ? iz : (d == 1 ? iy : ix);
    const int n = d == 0 ? g.nz : (d == 1 ? g.ny : g.nx);
    int sb;
    if (i >= -M && i < 0) sb = i + M;
    else if (i >= n && i < n + M) sb = M + (i - n);
    else return -1;
    if (d != 0 && (iz < 0 || iz >= g.nz)) return -1;
    if (d != 1 && (iy < 0 || iy >= g.ny)) return -1;
    if (d != 2 && (ix < 0 || ix >= g.nx)) return -1;
    if (d == 2) return ((long long)iz * g.ny + iy) * (2 * M) + sb;
    long long base = 2LL * M * g.nz * g.ny;
    if (d == 1) return base + ((long long)iz * (2 * M) + sb) * g.nx + ix;
    base += 2LL * M * g.nz * g.nx;
    return base + ((long long)sb * g.ny + iy) * g.nx + ix;
}

template <int M>
struct AdjSmem {
    using G = Geo<M>;
    static constexpr unsigned PA = 0;                                  // (p, lp) row z+W-1, core
    static constexpr unsigned LA = PA + al128(TX * TY * 8);            // lpsi_vz, row z+W-1 (strip)
    static constexpr unsigned VZ = LA + al128(TX * TY * 4);            // (vz, lvz) half row z+M-1
    static constexpr unsigned BK = VZ + al128(TX * TY * 8);            // 1/rho, row z+M
    static constexpr unsigned PZ = BK + al128(TX * TY * 4);            // lpsi_pz half row z+M-1 (strip)
    static constexpr unsigned PW = PZ + al128(TX * TY * 4);            // (p, lp) row z, wide
    static constexpr unsigned KW = PW + al128(G::XW2 * G::YH2 * 8);    // kdt row z, wide
    static constexpr unsigned LX = KW + al128(G::XW2 * G::YH2 * 4);    // lpsi_vx, x-wide (strip tiles)
    static constexpr unsigned LY = LX + al128(G::XW2 * TY * 4);        // lpsi_vy, y-wide (strip tiles)
    static constexpr unsigned VX = LY + al128(TX * G::YH2 * 4);        // (vx, lvx) xbox
    static constexpr unsigned VY = VX + al128(G::XW1 * TY * 8);        // (vy, lvy) ybox
    static constexpr unsigned BB = VY + al128(TX * G::YH1 * 8);        // 1/rho ybr
    static constexpr unsigned QX = BB + al128(G::XW1 * G::YHB * 4);    // lpsi_px xbox (strip tiles)
    static constexpr unsigned QY = QX + al128(G::XW1 * TY * 4);        // lpsi_py ybox (strip tiles)
    static constexpr unsigned STAGE = QY + al128(TX * G::YH1 * 4);
    static constexpr unsigned OWX = PD * STAGE;                        // (v^{n+1/2}, w) x half nodes
    static constexpr unsigned ONX = OWX + al128(G::XW1 * TY * 8);      // v^{n-1/2} x
    static constexpr unsigned OIX = ONX + al128(G::XW1 * TY * 4);      // G lambda_v products x
    static constexpr unsigned OWY = OIX + al128(G::XW1 * TY * 4);
    static constexpr unsigned ONY = OWY + al128(TX * G::YH1 * 8);
    static constexpr unsigned OIY = ONY + al128(TX * G::YH1 * 4);
    static constexpr unsigned BAR = OIY + al128(TX * G::YH1 * 4);
    static constexpr unsigned TOTAL = BAR + 64 + 128;
};

// two CTAs of each fused kernel per SM: 228 KB per SM, 1 KB reserved per CTA
static_assert(2 * (AdjSmem<4>::TOTAL + 1024) <= 233472 && 2 * (BornSmem<4>::TOTAL + 1024) <= 233472,
              "fused 3D kernels must fit two CTAs per SM");

}  // namespace

size_t fused3d_adj_smem(int M) { return M == 2 ? AdjSmem<2>::TOTAL : AdjSmem<4>::TOTAL; }

namespace {

template <int M>
__device__ __forceinline__ void adj_issue(const Adj3F &a, unsigned char *st, uint64_t *bar, int slot, int x0, int y0,
                                          int z, int zc0, bool px, bool py, bool px2, bool py2)
{
    using G = Geo<M>;
    using S = AdjSmem<M>;
    const GridDev &g = a.g;
    const int k = z + M - 1, r = z + G::W - 1;
    const bool main = z >= zc0;
    const bool rs = r >= 0 && r < g.Nz && (r <= g.z0 - 1 || r >= g.z0 + g.nz);   // node z strip
    const bool ks = k >= 0 && k < g.Nz && (k <= g.z0 - 2 || k >= g.z0 + g.nz);   // half-node z strip
    const int qp = slot * (a.in_planes / 2), qf = slot * a.in_planes;
    constexpr unsigned C8 = TX * TY * 8, C4 = TX * TY * 4;
    unsigned bytes = C8 + C8 + C4 + (rs ? C4 : 0) + (ks ? C4 : 0);
    if (main) {
        bytes += G::XW2 * G::YH2 * 12 + G::XW1 * TY * 8 + TX * G::YH1 * 8 + G::XW1 * G::YHB * 4;
        if (px2) bytes += G::XW2 * TY * 4;
        if (py2) bytes += TX * G::YH2 * 4;
        if (px) bytes += G::XW1 * TY * 4;
        if (py) bytes += TX * G::YH1 * 4;
    }
    const int xc = x0, x1 = x0 - G::XO1, x2 = x0 - G::XO2;   // floats; pairs use 2x
    if ((xc | x1 | x2) & 3) {
        atomicOr(a.err, 2);
        return;
    }
    mbar_expect(bar, bytes);
    tma4(st + S::PA, a.p_core, 2 * xc, y0, node_src_row(g, r), qp + A3F_PL / 2, bar);
    if (rs) tma4(st + S::LA, a.f_core, xc, y0, r, qf + A3F_LPVZ, bar);
    tma4(st + S::VZ, a.p_core, 2 * xc, y0, half_src_row(g, k), qp + A3F_VZ / 2, bar);
    tma4(st + S::BK, a.m_core, xc, y0, k + 1, 1, bar);
    if (ks) tma4(st + S::PZ, a.f_core, xc, y0, k, qf + A3F_LPPZ, bar);
    if (main) {
        tma4(st + S::PW, a.p_wide, 2 * x2, y0 - G::YO2, z, qp + A3F_PL / 2, bar);
        tma4(st + S::KW, a.m_wide, x2, y0 - G::YO2, z, 0, bar);
        if (px2) tma4(st + S::LX, a.f_xwide, x2, y0, z, qf + A3F_LPVX, bar);
        if (py2) tma4(st + S::LY, a.f_ywide, xc, y0 - G::YO2, z, qf + A3F_LPVY, bar);
        tma4(st + S::VX, a.p_xbox, 2 * x1, y0, z, qp + A3F_VX / 2, bar);
        tma4(st + S::VY, a.p_ybox, 2 * xc, y0 - G::YO1, z, qp + A3F_VY / 2, bar);
        tma4(st + S::BB, a.m_ybr, x1, y0 - G::YO1, z, 1, bar);
        if (px) tma4(st + S::QX, a.f_xbox, x1, y0, z, qf + A3F_LPPX, bar);
        if (py) tma4(st + S::QY, a.f_ybox, xc, y0 - G::YO1, z, qf + A3F_LPPY, bar);
    }
}

template <int M>
__global__ void __launch_bounds__(NTH, kMinBlocks) k3f_adj(const __grid_constant__ Adj3F a)
{
    if (guard_tripped(a.g)) return;
    using G = Geo<M>;
    using S = AdjSmem<M>;
    constexpr int W = G::W;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((128u - (su32(smem_raw) & 127u)) & 127u);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + S::BAR);
    float2 *oWX = reinterpret_cast<float2 *>(sm + S::OWX);
    float *oNX = reinterpret_cast<float *>(sm + S::ONX);
    float *oIX = reinterpret_cast<float *>(sm + S::OIX);
    float2 *oWY = reinterpret_cast<float2 *>(sm + S::OWY);
    float *oNY = reinterpret_cast<float *>(sm + S::ONY);
    float *oIY = reinterpret_cast<float *>(sm + S::OIY);

    const GridDev &g = a.g;
    const int t = threadIdx.x, tx = t % TX, ty = t / TX;
    const int nzc = (g.Nz + a.tzc - 1) / a.tzc;
    const int slot = blockIdx.z / nzc, zcn = blockIdx.z - slot * nzc;
    const int shot = a.shot0 + slot;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool colok = x < g.Nx && y < g.Ny;
    const int zc0 = zcn * a.tzc, zc1 = min(zc0 + a.tzc, g.Nz);
    const int zstart = zc0 - W;
    const float dt = g.dt;
    const int n = a.n;
    const bool recon = n > 0;
    const int pl = (int)g.plane, rowz = (int)g.rowz, pitch = g.pitch;
    const int cxy = y * pitch + x;
    const int ixg = x - g.x0, iyg = y - g.y0;
    const bool xin = ixg >= 0 && ixg < g.nx, yin = iyg >= 0 && iyg < g.ny;
    // CTA-uniform strip flags: half-node halos (px, py), node halos (px2, py2)
    const bool px = (x0 - M <= g.x0 - 2) || (x0 + TX + M - 2 >= g.x0 + g.nx);
    const bool py = (y0 - M <= g.y0 - 2) || (y0 + TY + M - 2 >= g.y0 + g.ny);
    const bool px2 = (x0 - 2 * M + 1 <= g.x0 - 1) || (x0 + TX + 2 * M - 2 >= g.x0 + g.nx);
    const bool py2 = (y0 - 2 * M + 1 <= g.y0 - 1) || (y0 + TY + 2 * M - 2 >= g.y0 + g.ny);
    const float *in = a.in + (long long)slot * a.in_planes * g.plane;
    float *outf = a.out + (long long)slot * a.out_planes * g.plane;
    float2 *out2 = reinterpret_cast<float2 *>(outf);
    float2 *img = a.img + (long long)slot * g.plane;
    const long long rowprev = band_row(a.bands, shot, n - 1);
    const int src = a.src_cell[shot];
    const float wsrc = recon ? a.src_scale * a.wav[(a.wav_per_shot ? (long long)shot * g.nt : 0) + n - 1] : 0.f;

    if (t == 0) {
        for (int i = 0; i < PD; ++i) mbar_init(bar + i);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (t == 0) {
        for (int j = 0; j < PD - 1; ++j)
            if (zstart + j < zc1)
                adj_issue<M>(a, sm + j * S::STAGE, bar + j, slot, x0, y0, zstart + j, zc0, px, py, px2, py2);
    }

    // (p^n, u_z) at node row rr of this column
    // (pq holds the mirror row's values for a ghost row rr < z0; the surface
    // row carries p = 0 and lambda_p = 0)
    auto pu_node = [&](int rr, float2 pq, float kd, float lpvz) -> float2 {
        if (g.fs && rr <= g.z0) return rr == g.z0 ? make_float2(0.f, 0.f) : make_float2(-pq.x, -(kd * pq.y));
        float u = kd * pq.y;
        if (colok && rr >= 0 && rr < g.Nz && (rr <= g.z0 - 1 || rr >= g.z0 + g.nz)) u -= a.pml.ai[0][rr] * (lpvz - u);
        return make_float2(pq.x, u);
    };
    // z rings: PU[m] node row z + m; VW, VN, PIZ half row z + m - M
    float2 PU[W], VW[W];
    float VN[W], PIZ[W];
#pragma unroll
    for (int m = 0; m < W; ++m) {
        VW[m] = make_float2(0.f, 0.f);
        VN[m] = 0.f;
        PIZ[m] = 0.f;
    }
    {
        const float2 *pin = reinterpret_cast<const float2 *>(in) + (A3F_PL / 2) * (long long)pl;
#pragma unroll
        for (int m = 0; m < W - 1; ++m) {
            const int rr = zstart + m, rs = node_src_row(g, rr);
            const bool ok = colok && rr >= 0 && rr < g.Nz;
            const int c = ok ? rr * rowz + cxy : 0;
            const float2 pq = (colok && rs >= 0 && rs < g.Nz) ? pin[rs * rowz + cxy] : make_float2(0.f, 0.f);
            const float kd = ok ? a.kdt[c] : 0.f;
            const float lv = (ok && (rr <= g.z0 - 1 || rr >= g.z0 + g.nz)) ? in[A3F_LPVZ * (long long)pl + c] : 0.f;
            PU[m] = pu_node(rr, pq, kd, lv);
        }
    }
    float bz_old = 0.f;
    {
        const int kk = zstart + M - 1;
        if (colok && kk >= 0 && kk < g.Nz) bz_old = a.binv[kk * rowz + cxy];
    }
    // dt kappa of the look-ahead node row, loaded one row ahead
    auto kd_at = [&](int rr) { return (colok && rr >= 0 && rr < g.Nz) ? a.kdt[rr * rowz + cxy] : 0.f; };
    float kd_r = kd_at(zstart + W - 1);

    bool failed = false;
    int fail_row = 0;
    for (int z = zstart; z < zc1; ++z) {
        const int j = z - zstart;
        const bool to = !mbar_wait(bar + j % PD, (unsigned)(j / PD) & 1u);
        if (__syncthreads_or(to)) {
            failed = true;
            fail_row = z;
            break;
        }
        if (t == NTH - 1 && z + PD - 1 < zc1) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            adj_issue<M>(a, sm + ((j + PD - 1) % PD) * S::STAGE, bar + (j + PD - 1) % PD, slot, x0, y0, z + PD - 1,
                         zc0, px, py, px2, py2);
        }
        unsigned char *st = sm + (j % PD) * S::STAGE;
        const int k = z + M - 1, r = z + W - 1;
        {
            const float2 pq = reinterpret_cast<const float2 *>(st + S::PA)[t];
            const bool rs = r >= 0 && r < g.Nz && (r <= g.z0 - 1 || r >= g.z0 + g.nz);
            PU[W - 1] = pu_node(r, pq, kd_r, rs ? reinterpret_cast<const float *>(st + S::LA)[t] : 0.f);
            kd_r = kd_at(r + 1);
        }
        // ---- half row k along z: lambda_vz, lambda_psi_pz, background vz^{n-1/2}
        {
            const float2 v2 = reinterpret_cast<const float2 *>(st + S::VZ)[t];
            const float bk1 = k + 1 < g.Nz ? reinterpret_cast<const float *>(st + S::BK)[t] : bz_old;
            float wz = 0.f, vn = 0.f, piz = 0.f;
            if (colok && k >= 0 && k < g.Nz) {
                const bool own = k >= zc0 && k < zc1;
                const int ck = k * rowz + cxy;
                const float2 D = st2<M>(g.cz, [&](int l) { return PU[M - 1 + l]; }, [&](int l) { return PU[M - l]; });
                const float lv = v2.y + D.y;
                const float dtbu = dt * 0.5f * (bz_old + bk1);
                wz = dtbu * lv;
                if (k <= g.z0 - 2 || k >= g.z0 + g.nz) {
                    const float l1 = reinterpret_cast<const float *>(st + S::PZ)[t] - dtbu * lv;
                    wz -= a.pml.ah[0][k] * l1;
                    if (own) outf[A3F_LPPZ * pl + ck] = a.pml.bh[0][k] * l1;
                }
                piz = D.x * lv;
                if (recon && xin && yin) {
                    const int iz = k - g.z0;
                    if ((iz >= 0 || g.fs) && iz < g.nz) vn = v2.x + dtbu * D.x;   // ghost half rows: mirrors
                    else {
                        const long long b = fband(g, 0, iz, iyg, ixg);
                        if (b >= 0) vn = band_get(a.bands, 1, rowprev, b);
                    }
                }
                if (own) out2[(A3F_VZ / 2) * pl + ck] = make_float2(vn, lv);
            }
            bz_old = bk1;
            VW[W - 1] = make_float2(v2.x, wz);
            VN[W - 1] = vn;
            PIZ[W - 1] = piz;
        }

        if (z >= zc0) {
            float2 *wP = reinterpret_cast<float2 *>(st + S::PW);
            const float *wK = reinterpret_cast<const float *>(st + S::KW);
            const float *bLX = reinterpret_cast<const float *>(st + S::LX);
            const float *bLY = reinterpret_cast<const float *>(st + S::LY);
            const float2 *bVX = reinterpret_cast<const float2 *>(st + S::VX);
            const float2 *bVY = reinterpret_cast<const float2 *>(st + S::VY);
            const float *bBB = reinterpret_cast<const float *>(st + S::BB);
            const float *bQX = reinterpret_cast<const float *>(st + S::QX);
            const float *bQY = reinterpret_cast<const float *>(st + S::QY);
            const int rz = z * rowz;
            // ---- (p, lambda_p) -> (p, dt kappa lambda_p) over the wide tile;
            // the thread's own node first (it keeps p^n and lambda_p)
            const int own_w = (ty + G::YO2) * G::XW2 + tx + G::XO2;
            const bool surf = g.fs && z == g.z0;   // free-surface row: p = 0, lambda_p = 0
            const float lsc = surf ? 0.f : 1.f;
            float2 pl1 = wP[own_w];
            pl1.y *= lsc;
            const float kd = wK[own_w];
            const float kl = kd * pl1.y;
            wP[own_w] = make_float2(pl1.x, kl);
            for (int i = t; i < G::XW2 * G::YH2; i += NTH) {
                const int rr = i / G::XW2, cc = i - rr * G::XW2;
                if (rr >= G::YO2 && rr < G::YO2 + TY && cc >= G::XO2 && cc < G::XO2 + TX) continue;
                const float2 v = wP[i];
                wP[i] = make_float2(v.x, wK[i] * (v.y * lsc));
            }
            // these generic-proxy writes to the stage must be ordered before the
            // TMA copy that refills it (issued after the next row's barrier):
            // every writing thread fences its own writes
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            // ---- half nodes on the x and y halos of the row
            constexpr int NVX = TY * G::NXI, NIT = NVX + G::YH1 * TX;
            for (int i = t; i < NIT; i += NTH) {
                if (i < NVX) {
                    const int iy = i / G::NXI, jx = i - iy * G::NXI;
                    const int xh = x0 - M + jx, yy = y0 + iy;
                    float2 vw = make_float2(0.f, 0.f);
                    float vn = 0.f, pi = 0.f;
                    const int cb = iy * G::XW1 + jx - M + G::XO1;   // xbox entry of half node xh
                    if (xh >= 0 && xh < g.Nx && yy < g.Ny) {
                        const int c0 = (iy + G::YO2) * G::XW2 + (jx - M + G::XO2);   // wide entry of node xh
                        const int l0 = iy * G::XW2 + (jx - M + G::XO2);              // x-wide entry of node xh
                        auto tap = [&](int l) -> float2 {
                            float2 v = wP[c0 + l];
                            if (px2) {
                                const int xn = xh + l;
                                if (xn >= 0 && xn < g.Nx && (xn <= g.x0 - 1 || xn >= g.x0 + g.nx))
                                    v.y -= a.pml.ai[2][xn] * (bLX[l0 + l] - v.y);
                            }
                            return v;
                        };
                        const float2 D = st2<M>(g.cx, [&](int l) { return tap(l); }, [&](int l) { return tap(1 - l); });
                        const float2 v2 = bVX[cb];
                        const float lv = v2.y + D.y;
                        const float b0 = bBB[M * G::XW1 + cb];
                        const float b1 = xh + 1 >= g.Nx ? b0 : bBB[M * G::XW1 + cb + 1];
                        const float dtbu = dt * 0.5f * (b0 + b1);
                        float w = dtbu * lv;
                        const bool own = jx >= M && jx < M + TX;
                        const int o = rz + yy * pitch + xh;
                        if (px && (xh <= g.x0 - 2 || xh >= g.x0 + g.nx)) {
                            const float l1 = bQX[cb] - dtbu * lv;
                            w -= a.pml.ah[2][xh] * l1;
                            if (own) outf[A3F_LPPX * pl + o] = a.pml.bh[2][xh] * l1;
                        }
                        pi = D.x * lv;
                        if (recon) {
                            const int iz = z - g.z0, iy2 = yy - g.y0, ix2 = xh - g.x0;
                            if (iz >= 0 && iz < g.nz && iy2 >= 0 && iy2 < g.ny) {
                                if (ix2 >= 0 && ix2 < g.nx) vn = v2.x + dtbu * D.x;
                                else {
                                    const long long b = fband(g, 2, iz, iy2, ix2);
                                    if (b >= 0) vn = band_get(a.bands, 1, rowprev, b);
                                }
                            }
                        }
                        if (own) out2[(A3F_VX / 2) * pl + o] = make_float2(vn, lv);
                        vw = make_float2(v2.x, w);
                    }
                    oWX[iy * G::XW1 + jx] = vw;
                    oNX[iy * G::XW1 + jx] = vn;
                    oIX[iy * G::XW1 + jx] = pi;
                } else {
                    const int i2 = i - NVX;
                    const int jy = i2 / TX, ix = i2 - jy * TX;
                    const int yh = y0 - M + jy, xx = x0 + ix;
                    float2 vw = make_float2(0.f, 0.f);
                    float vn = 0.f, pi = 0.f;
                    if (yh >= 0 && yh < g.Ny && xx < g.Nx) {
                        const int c0 = (jy + M - 1) * G::XW2 + ix + G::XO2;   // wide entry of node yh
                        const int l0 = (jy + M - 1) * TX + ix;                // y-wide entry of node yh
                        auto tap = [&](int l) -> float2 {
                            float2 v = wP[c0 + l * G::XW2];
                            if (py2) {
                                const int yn = yh + l;
                                if (yn >= 0 && yn < g.Ny && (yn <= g.y0 - 1 || yn >= g.y0 + g.ny))
                                    v.y -= a.pml.ai[1][yn] * (bLY[l0 + l * TX] - v.y);
                            }
                            return v;
                        };
                        const float2 D = st2<M>(g.cy, [&](int l) { return tap(l); }, [&](int l) { return tap(1 - l); });
                        const float2 v2 = bVY[i2];
                        const float lv = v2.y + D.y;
                        const float *bc = bBB + jy * G::XW1 + ix + G::XO1;
                        const float b0 = bc[0];
                        const float b1 = yh + 1 >= g.Ny ? b0 : bc[G::XW1];
                        const float dtbu = dt * 0.5f * (b0 + b1);
                        float w = dtbu * lv;
                        const bool own = jy >= M && jy < M + TY;
                        const int o = rz + yh * pitch + xx;
                        if (py && (yh <= g.y0 - 2 || yh >= g.y0 + g.ny)) {
                            const float l1 = bQY[i2] - dtbu * lv;
                            w -= a.pml.ah[1][yh] * l1;
                            if (own) outf[A3F_LPPY * pl + o] = a.pml.bh[1][yh] * l1;
                        }
                        pi = D.x * lv;
                        if (recon) {
                            const int iz = z - g.z0, iy2 = yh - g.y0, ix2 = xx - g.x0;
                            if (iz >= 0 && iz < g.nz && ix2 >= 0 && ix2 < g.nx) {
                                if (iy2 >= 0 && iy2 < g.ny) vn = v2.x + dtbu * D.x;
                                else {
                                    const long long b = fband(g, 1, iz, iy2, ix2);
                                    if (b >= 0) vn = band_get(a.bands, 1, rowprev, b);
                                }
                            }
                        }
                        if (own) out2[(A3F_VY / 2) * pl + o] = make_float2(vn, lv);
                        vw = make_float2(v2.x, w);
                    }
                    oWY[i2] = vw;
                    oNY[i2] = vn;
                    oIY[i2] = pi;
                }
            }
            __syncthreads();
            // ---- node of the thread's own column at row z
            if (colok) {
                const int hx = ty * G::XW1 + tx + M;     // x half node x (x + 1/2)
                const int hy = (ty + M) * TX + tx;       // y half node y
                const float2 Ex = st2<M>(g.cx, [&](int l) { return oWX[hx + l - 1]; }, [&](int l) { return oWX[hx - l]; });
                const float2 Ey = st2<M>(g.cy, [&](int l) { return oWY[hy + (l - 1) * TX]; },
                                         [&](int l) { return oWY[hy - l * TX]; });
                const float2 Ez = st2<M>(g.cz, [&](int l) { return VW[M + l - 1]; }, [&](int l) { return VW[M - l]; });
                const float2 E = add2(add2(Ex, Ey), Ez);   // (Q_n = D- . v^{n+1/2}, D- . w)
                const int c = rz + cxy;
                const int izg = z - g.z0;
                const bool inner = xin && yin && izg >= 0 && izg < g.nz;
                // D- . v^{n-1/2}, summed z, y, x as the background pass sums
                // it, so the rebuilt p^{n-1} undoes that pass's rounding
                float qn = 0.f;
                if (recon)
                    qn = (st1<M>(g.cz, [&](int l) { return VN[M + l - 1]; }, [&](int l) { return VN[M - l]; }) +
                          st1<M>(g.cy, [&](int l) { return oNY[hy + (l - 1) * TX]; },
                                 [&](int l) { return oNY[hy - l * TX]; })) +
                         st1<M>(g.cx, [&](int l) { return oNX[hx + l - 1]; }, [&](int l) { return oNX[hx - l]; });
                if (inner) {
                    float2 acc = img[c];
                    acc.x += E.x * pl1.y;
                    // (on the free surface the half row above is a ghost: no product of its own)
                    acc.y += (oIX[hx] + oIX[hx - 1]) + (oIY[hy] + oIY[hy - TX]) + (PIZ[M] + (surf ? 0.f : PIZ[M - 1]));
                    img[c] = acc;
                }
                float pn = 0.f;
                if (recon) {
                    if (inner) {
                        pn = pl1.x + kd * qn;
                        if (c == src) pn -= wsrc;
                    } else {
                        long long b = -1;
                        for (int d = 0; d < 3 && b < 0; ++d) b = fband(g, d, izg, iyg, ixg);
                        if (b >= 0) pn = band_get(a.bands, 0, rowprev, b);
                    }
                }
                out2[(A3F_PL / 2) * pl + c] =
                    (g.fs && z <= g.z0) ? make_float2(0.f, 0.f) : make_float2(pn, pl1.y + E.y);
                if (x <= g.x0 - 1 || x >= g.x0 + g.nx)
                    outf[A3F_LPVX * pl + c] = a.pml.bi[2][x] * (bLX[ty * G::XW2 + tx + G::XO2] - kl);
                if (y <= g.y0 - 1 || y >= g.y0 + g.ny)
                    outf[A3F_LPVY * pl + c] = a.pml.bi[1][y] * (bLY[(ty + G::YO2) * TX + tx] - kl);
                if (z <= g.z0 - 1 || z >= g.z0 + g.nz)
                    outf[A3F_LPVZ * pl + c] = a.pml.bi[0][z] * (in[A3F_LPVZ * pl + c] - kl);
            }
        }
#pragma unroll
        for (int m = 0; m < W - 1; ++m) {
            PU[m] = PU[m + 1];
            VW[m] = VW[m + 1];
            VN[m] = VN[m + 1];
            PIZ[m] = PIZ[m + 1];
        }
    }

    if (failed) {
        if (t == 0) {
            atomicOr(a.err, 1);
            const int jf = fail_row - zstart;
            for (int jj = jf; jj < jf + PD && zstart + jj < zc1; ++jj)
                (void)mbar_wait(bar + jj % PD, (unsigned)(jj / PD) & 1u);
        }
        return;
    }
    if (recon) {
        // pre-add the residual of step n-1 at the receivers of this tile
        __syncthreads();
        const int ntile = (int)(gridDim.x * gridDim.y) * nzc;
        const int tile = shot * ntile + (zcn * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        const int b = a.trec.ptr[tile], e = a.trec.ptr[tile + 1];
        for (int i = b + t; i < e; i += NTH) {
            const int2 rc = a.trec.rec[i];
            if (i > b && a.trec.rec[i - 1].x == rc.x) continue;   // run handled by its first entry
            float add = 0.f;
            for (int q = i; q < e && a.trec.rec[q].x == rc.x; ++q)
                add += a.dstage[(long long)a.trec.rec[q].y * g.nt + (n - 1)];
            out2[(A3F_PL / 2) * pl + rc.x].y += add;
        }
    }
}

// ---------------------------------------------------------------------------
// Tensor maps
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

}  // namespace

cudaError_t encode_tmap(CUtensorMap *m, CUtensorMapDataType type, int rank, const void *base, const cuuint64_t *dims,
                        const cuuint64_t *strides, const cuuint32_t *box)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(m, type, (cuuint32_t)rank, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor map over `nq` planes of `esz`-byte elements (4: float, 8: float2
// pair) starting at base: dims (x in floats, y, z, plane), box (bx elements,
// by rows, 1, 1); outside the padded grid the copy reads zeros.
cudaError_t make_tmap3(CUtensorMap *m, const void *base, const GridDev &g, int esz, long long nq, int bx, int by)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const int f = esz / 4;   // floats per element
    cuuint64_t dims[4] = {(cuuint64_t)g.Nx * f, (cuuint64_t)g.Ny, (cuuint64_t)g.Nz, (cuuint64_t)nq};
    cuuint64_t strides[3] = {(cuuint64_t)g.pitch * esz, (cuuint64_t)g.rowz * esz, (cuuint64_t)g.plane * esz};
    cuuint32_t box[4] = {(cuuint32_t)(bx * f), (cuuint32_t)by, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    if (((uintptr_t)base & 15) || box[0] > 256 || by > 256 || (box[0] * 4) % 16) return cudaErrorInvalidValue;
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Fills the tensor maps of a fused Born step reading `in` (pairs per slot
// in_pairs) with model pairs kd2 / br2.
cudaError_t fused3d_born_maps(Step3F &a, const float2 *kd2, const float2 *br2, int batch)
{
    const GridDev &g = a.g;
    cudaError_t e;
    const long long nq = (long long)batch * a.in_pairs;
    if (a.g.M == 2) {
        using G = Geo<2>;
        if ((e = make_tmap3(&a.in_wide, a.in, g, 8, nq, G::XW2, G::YH2)) != cudaSuccess) return e;
        if ((e = make_tmap3(&a.in_xbox, a.in, g, 8, nq, G::XW1, TY)) != cudaSuccess) return e;
        if ((e = make_tmap3(&a.in_ybox, a.in, g, 8, nq, TX, G::YH1)) != cudaSuccess) return e;
    } else {
        using G = Geo<4>;
        if ((e = make_tmap3(&a.in_wide, a.in, g, 8, nq, G::XW2, G::YH2)) != cudaSuccess) return e;
        if ((e = make_tmap3(&a.in_xbox, a.in, g, 8, nq, G::XW1, TY)) != cudaSuccess) return e;
        if ((e = make_tmap3(&a.in_ybox, a.in, g, 8, nq, TX, G::YH1)) != cudaSuccess) return e;
    }
    if ((e = make_tmap3(&a.in_core, a.in, g, 8, nq, TX, TY)) != cudaSuccess) return e;
    // model: plane 0 = kd2, plane 1 = br2 (one map over the two planes needs
    // them to be one plane apart)
    if (reinterpret_cast<const char *>(br2) - reinterpret_cast<const char *>(kd2) != (ptrdiff_t)(g.plane * 8))
        return cudaErrorInvalidValue;
    if ((e = make_tmap3(&a.m_core, kd2, g, 8, 2, TX, TY)) != cudaSuccess) return e;
    const int ybr = a.g.M == 2 ? Geo<2>::YHB : Geo<4>::YHB;
    return make_tmap3(&a.m_ybr, kd2, g, 8, 2, Geo<4>::XW1, ybr);
}

namespace {

// Start state of a fused reverse pass: pairs (p, 0), (vx, 0), (vy, 0), (vz, 0)
// from the saved background final state, whose planes are ordered
// [p][vz][vy][vx] (direction 0 = z in the background kernels).
__global__ void k3f_pack(const GridDev g, const float *final_state, int fs0, int batch, float *st,
                         long long sstride)
{
    const long long plane = g.plane;
    const long long n = batch * plane;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long s = i / plane, c = i - s * plane;
        const float *fs = final_state + (fs0 + s) * 4 * plane;
        float2 *o = reinterpret_cast<float2 *>(st + s * sstride);
        o[(A3F_PL / 2) * plane + c] = make_float2(fs[c], 0.f);
        o[(A3F_VZ / 2) * plane + c] = make_float2(fs[1 * plane + c], 0.f);
        o[(A3F_VY / 2) * plane + c] = make_float2(fs[2 * plane + c], 0.f);
        o[(A3F_VX / 2) * plane + c] = make_float2(fs[3 * plane + c], 0.f);
    }
}

}  // namespace

cudaError_t launch_pack3f(const GridDev &g, const float *final_state, int fs0, int batch, float *st,
                          long long sstride, cudaStream_t s)
{
    const long long n = batch * g.plane;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 16);
    k3f_pack<<<blocks, 256, 0, s>>>(g, final_state, fs0, batch, st, sstride);
    return cudaGetLastError();
}

cudaError_t fused3d_adj_maps(Adj3F &a, const float *kdt, const float *binv, int batch)
{
    const GridDev &g = a.g;
    cudaError_t e;
    const long long nqp = (long long)batch * (a.in_planes / 2), nqf = (long long)batch * a.in_planes;
    const bool m2 = g.M == 2;
    const int XW2 = m2 ? Geo<2>::XW2 : Geo<4>::XW2, YH2 = m2 ? Geo<2>::YH2 : Geo<4>::YH2;
    const int XW1 = Geo<4>::XW1, YH1 = m2 ? Geo<2>::YH1 : Geo<4>::YH1, YHB = m2 ? Geo<2>::YHB : Geo<4>::YHB;
    if ((e = make_tmap3(&a.p_core, a.in, g, 8, nqp, TX, TY)) != cudaSuccess) return e;
    if ((e = make_tmap3(&a.p_wide, a.in, g, 8, nqp, XW2, YH2)) != cudaSuccess) return e;
    if ((e = make_tmap3(&a.p_xbox, a.in, g, 8, nqp, XW1, TY)) != cudaSuccess) return e;
    if ((e = make_tmap3(&a.p_ybox, a.in, g, 8, nqp, TX, YH1)) != cudaSuccess) return e;
    if ((e = make_tmap3(&a.f_core, a.in, g, 4, nqf, TX, TY)) != cudaSuccess) return e;
    if ((e = make_tmap3(&a.f_xwide, a.in, g, 4, nqf, XW2, TY)) != cudaSuccess) return e;
    if ((e = make_tmap3(&a.f_ywide, a.in, g, 4, nqf, TX, YH2)) != cudaSuccess) return e;
    if ((e = make_tmap3(&a.f_xbox, a.in, g, 4, nqf, XW1, TY)) != cudaSuccess) return e;
    if ((e = make_tmap3(&a.f_ybox, a.in, g, 4, nqf, TX, YH1)) != cudaSuccess) return e;
    // model: plane 0 dt kappa, plane 1 1/rho (adjacent)
    if (binv - kdt != (ptrdiff_t)g.plane) return cudaErrorInvalidValue;
    if ((e = make_tmap3(&a.m_core, kdt, g, 4, 2, TX, TY)) != cudaSuccess) return e;
    if ((e = make_tmap3(&a.m_wide, kdt, g, 4, 2, XW2, YH2)) != cudaSuccess) return e;
    return make_tmap3(&a.m_ybr, kdt, g, 4, 2, XW1, YHB);
}

cudaError_t configure_3d_kernels()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k3f_born<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)BornSmem<2>::TOTAL)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k3f_born<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)BornSmem<4>::TOTAL)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k3f_adj<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)AdjSmem<2>::TOTAL)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k3f_adj<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AdjSmem<4>::TOTAL);
}

cudaError_t launch_adj3f(const Adj3F &a, int batch, cudaStream_t s)
{
    const GridDev &g = a.g;
    const int nzc = (g.Nz + a.tzc - 1) / a.tzc;
    dim3 grid((g.Nx + TX - 1) / TX, (g.Ny + TY - 1) / TY, nzc * batch);
    if (g.M == 2) k3f_adj<2><<<grid, NTH, AdjSmem<2>::TOTAL, s>>>(a);
    else k3f_adj<4><<<grid, NTH, AdjSmem<4>::TOTAL, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_born3f(const Step3F &a, int batch, cudaStream_t s)
{
    const GridDev &g = a.g;
    const int nzc = (g.Nz + a.tzc - 1) / a.tzc;
    dim3 grid((g.Nx + TX - 1) / TX, (g.Ny + TY - 1) / TY, nzc * batch);
    if (g.M == 2) k3f_born<2><<<grid, NTH, BornSmem<2>::TOTAL, s>>>(a);
    else k3f_born<4><<<grid, NTH, BornSmem<4>::TOTAL, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lsrtm
