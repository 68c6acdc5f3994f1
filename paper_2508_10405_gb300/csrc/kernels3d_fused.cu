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

namespace lsrtm {
namespace {

constexpr int TX = kTile3X, TY = kTile3Y, NTH = TX * TY;
constexpr int PD = 2;                       // stage ring depth
constexpr int kMinBlocks = 2;               // resident CTAs per SM the register budget targets
constexpr unsigned kWaitLimit = 1u << 22;   // mbarrier polls before giving up

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

// ---- shared memory, mbarriers and TMA
__device__ __forceinline__ unsigned su32(const void *p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t *b)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, unsigned phase)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase `phase` of barrier b; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned phase)
{
    for (unsigned i = 0; i < kWaitLimit; ++i)
        if (mbar_test(b, phase)) return true;
    return false;
}
__device__ __forceinline__ void tma4(void *dst, const CUtensorMap &m, int x, int y, int z, int q, uint64_t *b)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(&m)), "r"(x), "r"(y), "r"(z), "r"(q), "r"(su32(b))
        : "memory");
}

constexpr unsigned al128(unsigned b) { return (b + 127u) / 128u * 128u; }

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
    tma4(st + S::PA, a.in_core, xc, y0, r, q + F3_P, bar);
    tma4(st + S::VZ, a.in_core, xc, y0, k, q + F3_VZ, bar);
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
            const int zr = zstart + m;
            P[m] = (colok && zr >= 0 && zr < g.Nz) ? pin[zr * g.rowz + cxy] : make_float2(0.f, 0.f);
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
        P[W - 1] = cPA[t];
        const float2 brk1 = cBK[t];
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

cudaError_t configure_3d_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k3f_born<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)BornSmem<2>::TOTAL);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k3f_born<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BornSmem<4>::TOTAL);
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
