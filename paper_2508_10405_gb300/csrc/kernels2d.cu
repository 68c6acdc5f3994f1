// Fused 2D time-step kernels for the staggered-grid Born operator and its
// exact transpose (Eq. 1, Eq. scattereqln, App. A).
//
// One launch advances every shot of a batch by one time step. A CTA of 256
// threads owns one x-column per thread (240 output columns plus 2M halo
// columns on each side for M = 4) and marches down a z-chunk of the padded
// grid:
//   * along z the stencil operands live in per-thread register rings of
//     length 2M plus a group of look-ahead entries (the march is unrolled by
//     one group of rows and the rings shift after every group);
//   * along x each row passes through one shared-memory row per field;
//   * the global loads of row z + PD - 1 are issued as asynchronous copies
//     (cp.async, zero-filled out of range) into a PD-deep shared-memory stage
//     ring while row z is computed;
//   * a background field and its partner (the scattered field in Born
//     modelling, the adjoint field in migration) are interleaved as float2 in
//     HBM, so one 8-byte access and one packed FP32x2 FMA (FFMA2) serve both.
// For every row the velocity stage (half nodes) is computed on the output
// columns and the x halo, then the pressure stage (integer nodes), so a time
// step needs no grid-wide barrier. Inputs and outputs are separate (ping-pong)
// buffers; each state field is read once and written once per step from HBM.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "lsrtm_internal.cuh"
#include "tma.cuh"

namespace lsrtm {
namespace {

constexpr int NTH = kThreads2D;
constexpr int PDF = 4;   // depth of the asynchronous row pipeline (forward)
constexpr int PDA = 3;   // depth of the asynchronous row pipeline (adjoint; 3 CTAs per SM fit)
constexpr int kFwdMinBlocks = 2;   // resident CTAs per SM the register budget targets
constexpr int kFwdTMinBlocks = 3;  // the TMA-staged Born kernel: three CTAs per SM (measured +25%)
constexpr int kFwdPlainMinBlocks = 3;   // the background step without bands or pseudo-Hessian (modelling)
constexpr int kAdjMinBlocks = 3;
constexpr int kAdjMinBlocksFS = 2;   // the free-surface variant needs more registers
// The z-marches are unrolled by 2M / k*GroupDiv rows and shift their register
// rings after every group: a full 2M-row unroll made the migration loop body
// large enough to miss in the instruction cache.
constexpr int kAdjGroupDiv = 4;
constexpr int kFwdGroupDiv = 2;

// State layouts, as offsets in float planes within a shot slot.
// Born: float2 pairs (background, scattered).
enum { B_P = 0, B_VX = 2, B_VZ = 4, B_PPX = 6, B_PPZ = 8 };
enum { B_PVX = 0, B_PVZ = 2 };                 // in-place node CPML memories
// Background only (band saving, pseudo-Hessian): float.
enum { G_P = 0, G_VX = 1, G_VZ = 2, G_PPX = 3, G_PPZ = 4 };
enum { G_PVX = 0, G_PVZ = 1 };
// Adjoint: float2 pairs (background, lambda) and float lambda CPML memories.
enum { A_PL = 0, A_VX = 2, A_VZ = 4, A_LPPX = 6, A_LPPZ = 7, A_LPVX = 8, A_LPVZ = 9 };
// Slots of aperture-windowed shots carry the window's own model after the
// state: dt kappa and 1/rho (float planes), and the Born pairs (float2).
enum { W_KDT = 10, W_BINV = 11, W_KD2 = 12, W_BR2 = 14 };
static_assert(W_BR2 + 2 == kWinStatePlanes2D, "window slot layout");

// ---- packed arithmetic for T = float or float2
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 fma_(float a, float2 b, float2 c) { return __ffma2_rn(f2(a), b, c); }
__device__ __forceinline__ float add_(float a, float b) { return a + b; }
__device__ __forceinline__ float2 add_(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float mul_(float a, float b) { return a * b; }
__device__ __forceinline__ float2 mul_(float a, float2 b) { return __fmul2_rn(f2(a), b); }
template <class T> __device__ __forceinline__ T zero_();
template <> __device__ __forceinline__ float zero_<float>() { return 0.f; }
template <> __device__ __forceinline__ float2 zero_<float2>() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ float sub_(float a, float b) { return a - b; }
__device__ __forceinline__ float2 sub_(float2 a, float2 b) { return __ffma2_rn(f2(-1.f), b, a); }
__device__ __forceinline__ float neg_(float a) { return -a; }
__device__ __forceinline__ float2 neg_(float2 a) { return make_float2(-a.x, -a.y); }

// Free surface (method of images about row z0): a ghost node row r < z0
// reads its mirror row with the sign flipped (p odd), a ghost half row k < z0
// its mirror half row (v_z even); other rows read themselves.
template <bool FS>
__device__ __forceinline__ int node_src_row(const GridDev &g, int r) { return (FS && r < g.z0) ? fs_node_row(g, r) : r; }
template <bool FS>
__device__ __forceinline__ int half_src_row(const GridDev &g, int k) { return (FS && k < g.z0) ? fs_half_row(g, k) : k; }

// Staggered first difference sum_l c_l (a_l - b_l): the M differences are
// independent, then one multiply-add chain of depth M (short critical path).
template <int M, class T, class FA, class FB>
__device__ __forceinline__ T stencil(const float *c, FA fa, FB fb)
{
    T d[M];
#pragma unroll
    for (int l = 0; l < M; ++l) d[l] = sub_(fa(l + 1), fb(l + 1));
    T acc = mul_(c[0], d[0]);
#pragma unroll
    for (int l = 1; l < M; ++l) acc = fma_(c[l], d[l], acc);
    return acc;
}
__device__ __forceinline__ float xof(float v) { return v; }
__device__ __forceinline__ float xof(float2 v) { return v.x; }
__device__ __forceinline__ float yof(float) { return 0.f; }
__device__ __forceinline__ float yof(float2 v) { return v.y; }

// ---- boundary bands
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

__device__ __forceinline__ bool in_xstrip(int ix, int M, int nx)
{
    return (ix >= -M && ix < 0) || (ix >= nx && ix < nx + M);
}

// Band slot of a node for the p band, -1 if the node is not in it.
__device__ __forceinline__ long long pband_index(int iz, int ix, int M, int nz, int nx)
{
    if (iz >= 0 && iz < nz) return in_xstrip(ix, M, nx) ? band_xstrip(iz, ix, M, nz, nx) : -1;
    if (ix >= 0 && ix < nx && in_xstrip(iz, M, nz)) return band_zstrip(iz, ix, M, nz, nx);
    return -1;
}


// ---- asynchronous copies (pred = false zero-fills the destination)
template <class T>
__device__ __forceinline__ void cpa(T *dst, const T *src, bool pred)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte copies");
    unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    int n = pred ? (int)sizeof(T) : 0;
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Copy only where the field is used (the forward kernel's CPML memories): the
// stage slot keeps stale data elsewhere, which no consumer reads (every
// consumer tests the same condition), and warps outside the strips issue
// nothing. (In the migration kernel the extra branches cost more registers
// than the skipped copies save.)
template <class T>
__device__ __forceinline__ void cpa_if(T *dst, const T *src, bool pred)
{
    if (pred) cpa(dst, src, true);
}

// Waits until at most PDN-1 of this thread's copy groups are pending.
template <int PDN>
__device__ __forceinline__ void cp_wait_row() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PDN - 1) : "memory"); }

template <int M>
struct Cols {
    static constexpr int W = 2 * M;            // ring length along z
    static constexpr int HXP = 2 * M;          // halo columns per side
    static constexpr int TXO = NTH - 2 * HXP;  // output columns per CTA
};

// Stage ring of the forward kernel: 8 fields of 8-byte slots per thread.
constexpr int kFwdSlots = 8;
constexpr size_t kFwdStageSlotBytes = (size_t)kFwdSlots * NTH * 8;
constexpr size_t kFwdStageBytes = PDF * kFwdStageSlotBytes;
// Stage ring of the adjoint kernel: 5 float2 fields then 9 float fields.
constexpr int kAdjF2 = 5, kAdjF1 = 9;
constexpr size_t kAdjStageFloats = (size_t)(2 * kAdjF2 + kAdjF1) * NTH;
constexpr size_t kAdjStageBytes = PDA * kAdjStageFloats * sizeof(float);

// ---------------------------------------------------------------------------
// Forward step from n to n+1. BORN: the background and the scattered field as
// float2 pairs (Eq. scattereqln driven by the background). Otherwise the
// background alone as float, with BANDS saving the boundary bands of p^n and
// v^{n+1/2} and HESS accumulating the pseudo-Hessian diagonal of App. B.
// ---------------------------------------------------------------------------
template <bool BORN>
struct FwdT {
    using T = typename std::conditional<BORN, float2, float>::type;   // state (pair)
    using R = typename std::conditional<BORN, float2, float>::type;   // (1/rho, rr) or 1/rho
    using K = typename std::conditional<BORN, float2, float>::type;   // (dt kappa, dt kappa dlnk) or dt kappa
};

template <bool BORN>
struct FwdRow {
    using T = typename FwdT<BORN>::T;
    using R = typename FwdT<BORN>::R;
    using K = typename FwdT<BORN>::K;
    T p;      // node row z + 2M - 1 (look-ahead of the z rings)
    T vz;     // half row k = z + M - 1
    T psz;    // psi_pz at half row k (CPML rows)
    T vx;     // row z
    T psx;    // psi_px at row z (CPML columns)
    R br1;    // 1/rho (, rr) at row k + 1
    R brz;    // 1/rho (, rr) at row z
    K kd;     // dt kappa (, dt kappa dlnk) at row z
};

template <int M, bool BORN, bool WIN, bool FS>
__device__ __forceinline__ void fwd_issue(char *st, const Step2D &a, const float *in, int xc, int z,
                                          int zc0, int zc1, bool colok, bool vxok, bool outcol,
                                          bool pmlxh)
{
    using T = typename FwdT<BORN>::T;
    using R = typename FwdT<BORN>::R;
    using K = typename FwdT<BORN>::K;
    const GridDev &g = a.g;
    const int pitch = g.pitch;
    const int W = 2 * M;
    char *sl = st + threadIdx.x * 8;
    const T *fin = reinterpret_cast<const T *>(in);
    const R *br = WIN ? reinterpret_cast<const R *>(in + (BORN ? W_BR2 : W_BINV) * g.plane)
                      : (BORN ? reinterpret_cast<const R *>(a.br2) : reinterpret_cast<const R *>(a.binv));
    const K *kk = WIN ? reinterpret_cast<const K *>(in + (BORN ? W_KD2 : W_KDT) * g.plane)
                      : (BORN ? reinterpret_cast<const K *>(a.kd2) : reinterpret_cast<const K *>(a.kdt));
    const int pT = (int)g.plane;   // cells per plane: the stride of one (pair) field in units of T (in-slot offsets fit 32 bits)
    const int oP = BORN ? B_P / 2 : G_P, oVX = BORN ? B_VX / 2 : G_VX, oVZ = BORN ? B_VZ / 2 : G_VZ;
    const int oPPX = BORN ? B_PPX / 2 : G_PPX, oPPZ = BORN ? B_PPZ / 2 : G_PPZ;
    const int zr = z + W - 1, k = z + M - 1;
    const int zrs = node_src_row<FS>(g, zr), ks = half_src_row<FS>(g, k);
    const bool okr = colok && zrs >= 0 && zrs < g.Nz;
    const int cr = okr ? zrs * pitch + xc : 0;
    const bool okk1 = colok && k + 1 >= 0;
    const int ck1 = okk1 ? min(k + 1, g.Nz - 1) * pitch + xc : 0;
    const bool okk = colok && k >= 0 && k < g.Nz;
    const int ck = okk ? k * pitch + xc : 0;
    const bool okks = okk && ks < g.Nz;
    const int cks = okks ? ks * pitch + xc : 0;
    const bool pz = okk && ((k <= g.z0 - 2) || (k >= g.z0 + g.nz));
    const bool main = z >= zc0 && z < zc1;
    const bool okz = colok && main;
    const int cz = okz ? z * pitch + xc : 0;
    const bool okv = vxok && main;
    const bool oko = outcol && main;
    constexpr size_t F = (size_t)NTH * 8;   // bytes between field rows of a stage
    cpa(reinterpret_cast<T *>(sl + 0 * F), fin + oP * pT + cr, okr);
    cpa(reinterpret_cast<T *>(sl + 1 * F), fin + oVZ * pT + cks, okks);
    cpa_if(reinterpret_cast<T *>(sl + 2 * F), fin + oPPZ * pT + ck, pz);
    cpa(reinterpret_cast<T *>(sl + 3 * F), fin + oVX * pT + cz, okv);
    cpa_if(reinterpret_cast<T *>(sl + 4 * F), fin + oPPX * pT + cz, okv && pmlxh);
    cpa(reinterpret_cast<R *>(sl + 5 * F), br + ck1, okk1);
    cpa(reinterpret_cast<R *>(sl + 6 * F), br + cz, okz);
    cpa(reinterpret_cast<K *>(sl + 7 * F), kk + cz, oko);
}

template <bool BORN>
__device__ __forceinline__ FwdRow<BORN> fwd_read(const char *st)
{
    using T = typename FwdT<BORN>::T;
    using R = typename FwdT<BORN>::R;
    using K = typename FwdT<BORN>::K;
    const char *sl = st + threadIdx.x * 8;
    constexpr size_t F = (size_t)NTH * 8;
    FwdRow<BORN> r;
    r.p = *reinterpret_cast<const T *>(sl + 0 * F);
    r.vz = *reinterpret_cast<const T *>(sl + 1 * F);
    r.psz = *reinterpret_cast<const T *>(sl + 2 * F);
    r.vx = *reinterpret_cast<const T *>(sl + 3 * F);
    r.psx = *reinterpret_cast<const T *>(sl + 4 * F);
    r.br1 = *reinterpret_cast<const R *>(sl + 5 * F);
    r.brz = *reinterpret_cast<const R *>(sl + 6 * F);
    r.kd = *reinterpret_cast<const K *>(sl + 7 * F);
    return r;
}

template <int M, bool BORN, bool BANDS, bool HESS, bool WIN, bool FS>
__global__ void __launch_bounds__(NTH, (BORN || BANDS || HESS) ? kFwdMinBlocks : kFwdPlainMinBlocks) k_fwd2d(const Step2D a)
{
    if (guard_tripped(a.g)) return;
    using C = Cols<M>;
    using T = typename FwdT<BORN>::T;
    using R = typename FwdT<BORN>::R;
    constexpr int W = C::W, HXP = C::HXP, TXO = C::TXO;
    __shared__ T sP[NTH];
    __shared__ R sB[NTH];
    __shared__ T sV[NTH];
    __shared__ float sH[HESS ? NTH : 1];
    extern __shared__ __align__(16) char stages[];   // [PDF][kFwdSlots][NTH] x 8 bytes

    const GridDev &g = a.g;
    const int t = threadIdx.x;
    const int slot = blockIdx.z, shot = a.shot0 + slot;
    // padded and interior widths of this shot's grid (its aperture window)
    const int Nx = WIN ? a.win_nx[shot] + 2 * g.x0 : g.Nx;
    const int nx = WIN ? Nx - 2 * g.x0 : g.nx;
    if (WIN && (int)blockIdx.x * TXO >= Nx) return;   // no output column in this shot's window
    const int x = (int)blockIdx.x * TXO - HXP + t;
    const bool colok = x >= 0 && x < Nx;
    const bool outcol = colok && t >= HXP && t < HXP + TXO;
    const bool vxok = colok && t >= M - 1 && t <= NTH - 1 - M;
    const int zc0 = (int)blockIdx.y * a.tzc;
    const int zc1 = min(zc0 + a.tzc, g.Nz);
    const int zstart = zc0 - W;
    const long long plane = g.plane;
    const int pT = (int)plane;   // in-slot offsets fit 32 bits (checked by the host)
    const int pitch = g.pitch;
    const int xc = colok ? x : 0;
    const float *in = a.in + slot * a.sstride;
    T *out = reinterpret_cast<T *>(a.out + slot * a.sstride) + xc;
    T *psiv = reinterpret_cast<T *>(a.psiv + slot * a.vstride) + xc;
    const float dt = g.dt;
    const int x0 = g.x0, x1 = g.x0 + nx, z0 = g.z0, z1 = g.z0 + g.nz;
    const int ix = x - x0;
    const bool pmlxh = colok && ((x <= x0 - 2) || (x >= x1));
    const bool pmlxn = colok && ((x <= x0 - 1) || (x >= x1));
    const int px = WIN ? shot * a.pml_xstride + x : x;   // x CPML profiles of this shot's window
    const float ahx = pmlxh ? a.pml.ah[2][px] : 0.f, bhx = pmlxh ? a.pml.bh[2][px] : 0.f;
    const float aix = pmlxn ? a.pml.ai[2][px] : 0.f, bix = pmlxn ? a.pml.bi[2][px] : 0.f;
    const long long bandoff = band_base(a.bands, shot, a.n);
    const int src = a.src_cell[shot];
    const float wsrc = a.src_scale * a.wav[(a.wav_per_shot ? (long long)shot * g.nt : 0) + a.n];
    constexpr int oP = BORN ? B_P / 2 : G_P, oVX = BORN ? B_VX / 2 : G_VX, oVZ = BORN ? B_VZ / 2 : G_VZ;
    constexpr int oPPX = BORN ? B_PPX / 2 : G_PPX, oPPZ = BORN ? B_PPZ / 2 : G_PPZ;
    constexpr int oPVX = BORN ? B_PVX / 2 : G_PVX, oPVZ = BORN ? B_PVZ / 2 : G_PVZ;

    // z rings, shifted by U entries after every group of U rows (entry u + m
    // holds row z + m of P, or the half-row value written m - W + 1 rows earlier)
    constexpr int U = W / kFwdGroupDiv > 0 ? W / kFwdGroupDiv : 1, RL = W + U - 1;
    T P[RL], VZ[RL];
    float HZ[HESS ? RL : 1];
#pragma unroll
    for (int j = 0; j < RL; ++j) {
        P[j] = zero_<T>();
        VZ[j] = zero_<T>();
        if (HESS) HZ[j] = 0.f;
    }
    {
        const T *pin = reinterpret_cast<const T *>(in) + oP * pT + xc;
#pragma unroll
        for (int j = 0; j < W - 1; ++j) {
            const int zr = zstart + j, zrs = node_src_row<FS>(g, zr);
            const T v = (colok && zrs >= 0 && zrs < g.Nz) ? pin[zrs * pitch] : zero_<T>();
            P[j] = zrs != zr ? neg_(v) : v;
        }
    }
    R br_old = zero_<R>();
    {
        const R *br = WIN ? reinterpret_cast<const R *>(in + (BORN ? W_BR2 : W_BINV) * plane)
                          : (BORN ? reinterpret_cast<const R *>(a.br2) : reinterpret_cast<const R *>(a.binv));
        int k = zstart + M - 1;
        if (colok && k >= 0 && k < g.Nz) br_old = br[k * pitch + xc];
    }

#pragma unroll
    for (int j = 0; j < PDF - 1; ++j) {
        if (zstart + j < zc1)
            fwd_issue<M, BORN, WIN, FS>(stages + j * kFwdStageSlotBytes, a, in, xc, zstart + j, zc0, zc1, colok, vxok,
                               outcol, pmlxh);
        cp_commit();
    }

    for (int zb = zstart; zb < zc1; zb += U) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int z = zb + u;
            if (z >= zc1) break;
            const int zi = z + PDF - 1;
            if (zi < zc1)
                fwd_issue<M, BORN, WIN, FS>(stages + ((zi - zstart) % PDF) * kFwdStageSlotBytes, a, in, xc, zi, zc0, zc1,
                                   colok, vxok, outcol, pmlxh);
            cp_commit();
            cp_wait_row<PDF>();
            const FwdRow<BORN> cur = fwd_read<BORN>(stages + ((z - zstart) % PDF) * kFwdStageSlotBytes);
            const int k = z + M - 1;   // half row of vz computed in this iteration
            const int sl = u + W - 1;
            P[sl] = (FS && z + W - 1 < g.z0) ? neg_(cur.p) : cur.p;   // ghost rows hold -p(mirror)
            // ---- vz at half row k (column-local)
            const float buz = 0.5f * (xof(br_old) + xof(cur.br1));
            const float rsum = yof(br_old) + yof(cur.br1);
            br_old = cur.br1;
            T vzn = zero_<T>();
            float hzq = 0.f;
            if (colok && k >= 0 && k < g.Nz) {
                const int ck = k * pitch;
                const bool own = outcol && k >= zc0 && k < zc1;
                T G = stencil<M, T>(g.cz, [&](int l) { return P[u + M - 1 + l]; },
                                    [&](int l) { return P[u + M - l]; });
                if ((k <= z0 - 2) || (k >= z1)) {
                    T ps = fma_(a.pml.bh[0][k], cur.psz, mul_(a.pml.ah[0][k], G));
                    if (own) out[oPPZ * pT + ck] = ps;
                    G = add_(G, ps);
                }
                const float dtbu = dt * buz;
                vzn = fma_(-dtbu, G, cur.vz);
                if constexpr (BORN) vzn.y = fmaf(0.5f * dt * rsum, G.x, vzn.y);
                if (own) {
                    out[oVZ * pT + ck] = vzn;
                    if (BANDS) {
                        int iz = k - z0;
                        if (ix >= 0 && ix < nx && in_xstrip(iz, M, g.nz))
                            band_put(a.bands, 1, slot, bandoff, band_zstrip(iz, ix, M, g.nz, nx), xof(vzn));
                    }
                }
                if (HESS) {
                    float q = buz * xof(G);
                    hzq = q * q;
                }
            }
            VZ[sl] = vzn;
            if (HESS) HZ[sl] = hzq;
            if (z < zc0) continue;   // warm-up rows of the z rings

            // ---- row z: vx on the output columns and the halo
            const int cz = z * pitch;
            const T p0 = P[u];
            sP[t] = p0;
            sB[t] = cur.brz;
            __syncthreads();
            T vxn = zero_<T>();
            float hxq = 0.f;
            if (vxok) {
                T G = stencil<M, T>(g.cx, [&](int l) { return sP[t + l]; }, [&](int l) { return sP[t + 1 - l]; });
                const bool last = x + 1 >= Nx;
                const R bn = last ? cur.brz : sB[t + 1];
                const float bux = 0.5f * (xof(cur.brz) + xof(bn));
                if (pmlxh) {
                    T ps = fma_(bhx, cur.psx, mul_(ahx, G));
                    if (outcol) out[oPPX * pT + cz] = ps;
                    G = add_(G, ps);
                }
                const float dtbu = dt * bux;
                vxn = fma_(-dtbu, G, cur.vx);
                if constexpr (BORN) {
                    float rs = yof(cur.brz) + (last ? 0.f : yof(bn));
                    vxn.y = fmaf(0.5f * dt * rs, G.x, vxn.y);
                }
                if (outcol) {
                    out[oVX * pT + cz] = vxn;
                    if (BANDS) {
                        int iz = z - z0;
                        if (iz >= 0 && iz < g.nz && in_xstrip(ix, M, nx))
                            band_put(a.bands, 1, slot, bandoff, band_xstrip(iz, ix, M, g.nz, nx), xof(vxn));
                    }
                }
                if (HESS) {
                    float q = bux * xof(G);
                    hxq = q * q;
                }
            }
            sV[t] = vxn;
            if (HESS) sH[t] = hxq;
            __syncthreads();

            // ---- row z: pressure on the output columns
            if (outcol) {
                T qx = stencil<M, T>(g.cx, [&](int l) { return sV[t + l - 1]; }, [&](int l) { return sV[t - l]; });
                T qz = stencil<M, T>(g.cz, [&](int l) { return VZ[u + M + l - 1]; },
                                     [&](int l) { return VZ[u + M - l]; });
                if (pmlxn) {
                    T ps = fma_(bix, psiv[oPVX * pT + cz], mul_(aix, qx));
                    psiv[oPVX * pT + cz] = ps;
                    qx = add_(qx, ps);
                }
                if ((z <= z0 - 1) || (z >= z1)) {
                    T ps = fma_(a.pml.bi[0][z], psiv[oPVZ * pT + cz], mul_(a.pml.ai[0][z], qz));
                    psiv[oPVZ * pT + cz] = ps;
                    qz = add_(qz, ps);
                }
                const T Q = add_(qx, qz);
                const float kd = xof(cur.kd);
                T pn = fma_(-kd, Q, p0);
                if constexpr (BORN) {
                    pn.y = fmaf(-cur.kd.y, Q.x, pn.y);
                    if (cz + x == src) pn.x += wsrc;
                } else {
                    if (cz + x == src) pn += wsrc;
                }
                if (FS && z <= z0) pn = zero_<T>();   // p = 0 on the free surface (ghost rows unused)
                out[oP * pT + cz] = pn;
                if (BANDS) {
                    long long b = pband_index(z - z0, ix, M, g.nz, nx);
                    if (b >= 0) band_put(a.bands, 0, slot, bandoff, b, xof(p0));
                }
                if (HESS) {
                    int iz = z - z0;
                    if (iz >= 0 && iz < g.nz && ix >= 0 && ix < nx) {
                        float bx0 = xof(cur.brz);
                        float hr = 0.5f * ((sH[t] + sH[t - 1]) + (HZ[u + M] + HZ[u + M - 1])) / (bx0 * bx0);
                        float kq = kd * xof(Q) / dt;
                        (a.hess + slot * plane)[cz + xc] += dt * (hr + kq * kq);
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < W - 1; ++j) {
            P[j] = P[j + U];
            VZ[j] = VZ[j + U];
            if (HESS) HZ[j] = HZ[j + U];
        }
    }

    if (BORN || a.rec_bg) {
        // record dp^{n+1} (Born) or the background p^{n+1} (nonlinear
        // modelling) at the receivers of this CTA
        __syncthreads();
        int tile = shot * a.trec.ntiles + blockIdx.y * gridDim.x + blockIdx.x;
        int b = a.trec.ptr[tile], e = a.trec.ptr[tile + 1];
        if constexpr (BORN) {
            const float2 *po = reinterpret_cast<const float2 *>(a.out + slot * a.sstride + B_P * plane);
            for (int i = b + t; i < e; i += NTH) {
                int2 rc = a.trec.rec[i];
                a.dstage[(long long)rc.y * g.nt + a.n] = a.rec_bg ? po[rc.x].x : po[rc.x].y;
            }
        } else {
            const float *po = a.out + slot * a.sstride + G_P * plane;
            for (int i = b + t; i < e; i += NTH) {
                int2 rc = a.trec.rec[i];
                a.dstage[(long long)rc.y * g.nt + a.n] = po[rc.x];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Born step with TMA row staging (shots without aperture windows): k_fwd2d's
// Born arithmetic in the same order, with the rows ahead staged as in
// k_adj2t (one thread issues each field row of a stage as one tile copy on
// the stage's mbarrier; zero fill outside the grid; unused fields not copied;
// a stage is refilled only after a barrier that follows every read of it).
// ---------------------------------------------------------------------------
struct Fwd2T {
    Step2D a;
    Maps2D m;
};

constexpr unsigned kFwdStageBytesT = (unsigned)kFwdStageSlotBytes;
static_assert(kFwdStageBytesT % 128 == 0, "stage rows stay 128-byte aligned");
constexpr unsigned kFwdBarOff = PDF * kFwdStageBytesT;
constexpr unsigned kFwdSmemT = kFwdBarOff + 64 + 128;   // stages, barriers, alignment slack

// Issues the copies of row z (the stage layout of fwd_issue) on barrier b;
// tph: the CTA has half-node CPML columns.
template <int M, bool FS>
__device__ __forceinline__ void fwd_issue_tma(const Fwd2T &p, char *st, uint64_t *b, int slot, int xs, int z,
                                              int zc0, int zc1, bool tph)
{
    const GridDev &g = p.a.g;
    const Maps2D &m = p.m;
    constexpr int W = 2 * M;
    constexpr unsigned F = NTH * 8;   // bytes of one field row
    const int zr = z + W - 1, k = z + M - 1;
    const int qp = slot * m.pps;
    const bool ink = k >= 0 && k < g.Nz;
    int rp = zr, rvz = ink ? k : -1;
    if constexpr (FS) {
        const int zrs = node_src_row<FS>(g, zr), ks = half_src_row<FS>(g, k);
        rp = (zrs >= 0 && zrs < g.Nz) ? zrs : -1;
        rvz = (ink && ks < g.Nz) ? ks : -1;
    }
    const int rb1 = k + 1 >= 0 ? min(k + 1, g.Nz - 1) : -1;
    const bool pz = ink && ((k <= g.z0 - 2) || (k >= g.z0 + g.nz));
    const bool main = z >= zc0 && z < zc1;
    const bool px = main && tph;
    const unsigned bytes = (3 + (pz ? 1 : 0) + (main ? 3 : 0) + (px ? 1 : 0)) * F;
    tma::fence_proxy_async();
    tma::mbar_expect(b, bytes);
    tma::load3(st + 0 * F, m.pr, xs, rp, qp + B_P / 2, b);
    tma::load3(st + 1 * F, m.pr, xs, rvz, qp + B_VZ / 2, b);
    if (pz) tma::load3(st + 2 * F, m.pr, xs, k, qp + B_PPZ / 2, b);
    tma::load3(st + 5 * F, m.mb, xs, rb1, 1, b);
    if (main) {
        tma::load3(st + 3 * F, m.pr, xs, z, qp + B_VX / 2, b);
        tma::load3(st + 6 * F, m.mb, xs, z, 1, b);
        tma::load3(st + 7 * F, m.mb, xs, z, 0, b);
    }
    if (px) tma::load3(st + 4 * F, m.pr, xs, z, qp + B_PPX / 2, b);
}

template <int M, bool FS>
__global__ void __launch_bounds__(NTH, kFwdTMinBlocks) k_fwd2t(const __grid_constant__ Fwd2T p)
{
    const Step2D &a = p.a;
    if (guard_tripped(a.g)) return;
    using C = Cols<M>;
    using T = float2;
    using R = float2;
    constexpr int W = C::W, HXP = C::HXP, TXO = C::TXO;
    static_assert(TXO % 2 == 0 && HXP % 2 == 0, "CTA column starts must be 16-byte aligned for 8-byte elements");
    __shared__ T sP[NTH];
    __shared__ R sB[NTH];
    __shared__ T sV[NTH];
    extern __shared__ unsigned char smraw[];
    unsigned char *sm = smraw + ((128u - (tma::su32(smraw) & 127u)) & 127u);
    char *stages = reinterpret_cast<char *>(sm);   // [PDF][kFwdSlots][NTH] x 8 bytes
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kFwdBarOff);

    const GridDev &g = a.g;
    const int t = threadIdx.x;
    const int slot = blockIdx.z, shot = a.shot0 + slot;
    const int Nx = g.Nx, nx = g.nx;
    const int xs = (int)blockIdx.x * TXO - HXP;
    const int x = xs + t;
    const bool colok = x >= 0 && x < Nx;
    const bool outcol = colok && t >= HXP && t < HXP + TXO;
    const bool vxok = colok && t >= M - 1 && t <= NTH - 1 - M;
    const int zc0 = (int)blockIdx.y * a.tzc;
    const int zc1 = min(zc0 + a.tzc, g.Nz);
    const int zstart = zc0 - W;
    const long long plane = g.plane;
    const int pT = (int)plane;   // in-slot offsets fit 32 bits (checked by the host)
    const int pitch = g.pitch;
    const int xc = colok ? x : 0;
    const float *in = a.in + slot * a.sstride;
    T *out = reinterpret_cast<T *>(a.out + slot * a.sstride) + xc;
    T *psiv = reinterpret_cast<T *>(a.psiv + slot * a.vstride) + xc;
    const float dt = g.dt;
    const int x0 = g.x0, x1 = g.x0 + nx, z0 = g.z0, z1 = g.z0 + g.nz;
    const bool pmlxh = colok && ((x <= x0 - 2) || (x >= x1));
    const bool pmlxn = colok && ((x <= x0 - 1) || (x >= x1));
    const bool tph = (xs <= x0 - 2) || (xs + NTH - 1 >= x1);   // CTA has half-node CPML columns
    const float ahx = pmlxh ? a.pml.ah[2][x] : 0.f, bhx = pmlxh ? a.pml.bh[2][x] : 0.f;
    const float aix = pmlxn ? a.pml.ai[2][x] : 0.f, bix = pmlxn ? a.pml.bi[2][x] : 0.f;
    const int src = a.src_cell[shot];
    const float wsrc = a.src_scale * a.wav[(a.wav_per_shot ? (long long)shot * g.nt : 0) + a.n];
    constexpr int oP = B_P / 2, oVX = B_VX / 2, oVZ = B_VZ / 2, oPPX = B_PPX / 2, oPPZ = B_PPZ / 2;
    constexpr int oPVX = B_PVX / 2, oPVZ = B_PVZ / 2;
    constexpr int PR = NTH - 1;   // the thread that issues the copies

    if (t == 0) {
        for (int i = 0; i < PDF; ++i) tma::mbar_init(bar + i);
        tma::mbar_init_fence();
    }
    __syncthreads();
    if (t == PR) {
        for (int j = 0; j < PDF - 1 && zstart + j < zc1; ++j)
            fwd_issue_tma<M, FS>(p, stages + j * kFwdStageBytesT, bar + j, slot, xs, zstart + j, zc0, zc1, tph);
    }

    constexpr int U = W / kFwdGroupDiv > 0 ? W / kFwdGroupDiv : 1, RL = W + U - 1;
    T P[RL], VZ[RL];
#pragma unroll
    for (int j = 0; j < RL; ++j) {
        P[j] = zero_<T>();
        VZ[j] = zero_<T>();
    }
    {
        const T *pin = reinterpret_cast<const T *>(in) + oP * pT + xc;
#pragma unroll
        for (int j = 0; j < W - 1; ++j) {
            const int zr = zstart + j, zrs = node_src_row<FS>(g, zr);
            const T v = (colok && zrs >= 0 && zrs < g.Nz) ? pin[zrs * pitch] : zero_<T>();
            P[j] = zrs != zr ? neg_(v) : v;
        }
    }
    R br_old = zero_<R>();
    {
        int k = zstart + M - 1;
        if (colok && k >= 0 && k < g.Nz) br_old = a.br2[k * pitch + xc];
    }

    bool bad = false;      // this thread's wait gave up
    int fail_row = zc1;    // first row whose stage was not consumed
    for (int zb = zstart; zb < zc1; zb += U) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int z = zb + u;
            if (z >= zc1) break;
            const int j = z - zstart;
            // refill the stage of row z - 1 with row z + PDF - 1: every thread
            // passed a barrier after reading it (the previous row's)
            const int zi = z + PDF - 1;
            if (t == PR && zi < zc1)
                fwd_issue_tma<M, FS>(p, stages + ((j + PDF - 1) % PDF) * kFwdStageBytesT, bar + (j + PDF - 1) % PDF,
                                     slot, xs, zi, zc0, zc1, tph);
            bad |= !tma::mbar_wait(bar + j % PDF, (unsigned)(j / PDF) & 1u);
            const FwdRow<true> cur = fwd_read<true>(stages + (j % PDF) * kFwdStageBytesT);
            const int k = z + M - 1;   // half row of vz computed in this iteration
            const int sl = u + W - 1;
            P[sl] = (FS && z + W - 1 < g.z0) ? neg_(cur.p) : cur.p;   // ghost rows hold -p(mirror)
            // ---- vz at half row k (column-local)
            const float buz = 0.5f * (xof(br_old) + xof(cur.br1));
            const float rsum = yof(br_old) + yof(cur.br1);
            br_old = cur.br1;
            T vzn = zero_<T>();
            if (colok && k >= 0 && k < g.Nz) {
                const int ck = k * pitch;
                const bool own = outcol && k >= zc0 && k < zc1;
                T G = stencil<M, T>(g.cz, [&](int l) { return P[u + M - 1 + l]; },
                                    [&](int l) { return P[u + M - l]; });
                if ((k <= z0 - 2) || (k >= z1)) {
                    T ps = fma_(a.pml.bh[0][k], cur.psz, mul_(a.pml.ah[0][k], G));
                    if (own) out[oPPZ * pT + ck] = ps;
                    G = add_(G, ps);
                }
                const float dtbu = dt * buz;
                vzn = fma_(-dtbu, G, cur.vz);
                vzn.y = fmaf(0.5f * dt * rsum, G.x, vzn.y);
                if (own) out[oVZ * pT + ck] = vzn;
            }
            VZ[sl] = vzn;
            if (z < zc0) {
                // warm-up row: the barrier that lets its stage be refilled
                if (__syncthreads_or(bad)) {
                    fail_row = z;
                    break;
                }
                continue;
            }

            // ---- row z: vx on the output columns and the halo
            const int cz = z * pitch;
            const T p0 = P[u];
            sP[t] = p0;
            sB[t] = cur.brz;
            if (__syncthreads_or(bad)) {
                fail_row = z;
                break;
            }
            T vxn = zero_<T>();
            if (vxok) {
                T G = stencil<M, T>(g.cx, [&](int l) { return sP[t + l]; }, [&](int l) { return sP[t + 1 - l]; });
                const bool last = x + 1 >= Nx;
                const R bn = last ? cur.brz : sB[t + 1];
                const float bux = 0.5f * (xof(cur.brz) + xof(bn));
                if (pmlxh) {
                    T ps = fma_(bhx, cur.psx, mul_(ahx, G));
                    if (outcol) out[oPPX * pT + cz] = ps;
                    G = add_(G, ps);
                }
                const float dtbu = dt * bux;
                vxn = fma_(-dtbu, G, cur.vx);
                float rs = yof(cur.brz) + (last ? 0.f : yof(bn));
                vxn.y = fmaf(0.5f * dt * rs, G.x, vxn.y);
                if (outcol) out[oVX * pT + cz] = vxn;
            }
            sV[t] = vxn;
            __syncthreads();

            // ---- row z: pressure on the output columns
            if (outcol) {
                T qx = stencil<M, T>(g.cx, [&](int l) { return sV[t + l - 1]; }, [&](int l) { return sV[t - l]; });
                T qz = stencil<M, T>(g.cz, [&](int l) { return VZ[u + M + l - 1]; },
                                     [&](int l) { return VZ[u + M - l]; });
                if (pmlxn) {
                    T ps = fma_(bix, psiv[oPVX * pT + cz], mul_(aix, qx));
                    psiv[oPVX * pT + cz] = ps;
                    qx = add_(qx, ps);
                }
                if ((z <= z0 - 1) || (z >= z1)) {
                    T ps = fma_(a.pml.bi[0][z], psiv[oPVZ * pT + cz], mul_(a.pml.ai[0][z], qz));
                    psiv[oPVZ * pT + cz] = ps;
                    qz = add_(qz, ps);
                }
                const T Q = add_(qx, qz);
                const float kd = xof(cur.kd);
                T pn = fma_(-kd, Q, p0);
                pn.y = fmaf(-cur.kd.y, Q.x, pn.y);
                if (cz + x == src) pn.x += wsrc;
                if (FS && z <= z0) pn = zero_<T>();   // p = 0 on the free surface (ghost rows unused)
                out[oP * pT + cz] = pn;
            }
        }
        if (fail_row < zc1) break;
#pragma unroll
        for (int j = 0; j < W - 1; ++j) {
            P[j] = P[j + U];
            VZ[j] = VZ[j + U];
        }
    }

    if (fail_row < zc1) {
        // a wait gave up: record it, let the copies in flight land (rows up to
        // fail_row + PDF - 1 were issued), return
        if (t == PR) {
            atomicOr(a.err, 1);
            for (int zz = fail_row; zz <= min(fail_row + PDF - 1, zc1 - 1); ++zz) {
                const int jj = zz - zstart;
                (void)tma::mbar_wait(bar + jj % PDF, (unsigned)(jj / PDF) & 1u);
            }
        }
        return;
    }

    // record dp^{n+1} (or the background p^{n+1} in nonlinear modelling) at
    // the receivers of this CTA
    __syncthreads();
    int tile = shot * a.trec.ntiles + blockIdx.y * gridDim.x + blockIdx.x;
    int b = a.trec.ptr[tile], e = a.trec.ptr[tile + 1];
    const float2 *po = reinterpret_cast<const float2 *>(a.out + slot * a.sstride + B_P * plane);
    for (int i = b + t; i < e; i += NTH) {
        int2 rc = a.trec.rec[i];
        a.dstage[(long long)rc.y * g.nt + a.n] = a.rec_bg ? po[rc.x].x : po[rc.x].y;
    }
}

// ---------------------------------------------------------------------------
// Reverse step n (n = nt-1 .. 0) of L^T. Input state: (background p^n,
// lambda_p) with the residual of step n already added, (v^{n+1/2}, lambda_v)
// and the lambda CPML memories. The step applies the transposed Born
// sub-steps (S4^T, S3^T on the half nodes from lambda_p; S2^T, S1^T on the
// nodes from lambda_v), accumulates the two zero-lag images (discrete
// transposed forms of Eqs. gradkappa, gradrho), rebuilds p^{n-1}, v^{n-1/2}
// in the interior from the saved boundary bands, and pre-adds the residual of
// step n-1. The D+ stencils of (p^n, u) and the D- stencils of (v^{n+1/2}, w)
// run as packed pairs.
// ---------------------------------------------------------------------------
struct AdjRow {
    float2 pl;      // node row r = z + 2M - 1: (p^n, lambda_p)
    float2 v2z;     // half row k: (vz^{n+1/2}, lambda_vz)
    float2 plz;     // row z: (p^n, lambda_p)
    float2 v2x;     // row z: (vx^{n+1/2}, lambda_vx)
    float2 img;     // row z: image accumulators
    float kdr, lpvzr, bz, lppz, kdz, lpsvx, lpsvz, bx, lppx;
};

template <int M, bool WIN, bool FS>
__device__ __forceinline__ void adj_issue(float *st, const Step2D &a, const float2 *img, const float *in,
                                          int xc, int z, int zc0, int zc1, bool colok, bool vxok,
                                          bool outcol, bool pmlxh, bool pmlxn, bool inner_col)
{
    const GridDev &g = a.g;
    const long long plane = g.plane;
    const long long p2 = plane;   // cells per plane: the stride of one pair field in float2 units
    const int pitch = g.pitch;
    const int W = 2 * M;
    const int z0 = g.z0, z1 = g.z0 + g.nz;
    const int t = threadIdx.x;
    float2 *s2 = reinterpret_cast<float2 *>(st) + t;
    float *s1 = st + 2 * kAdjF2 * NTH + t;
    const float2 *in2 = reinterpret_cast<const float2 *>(in);
    const int zr = z + W - 1, k = z + M - 1;
    const bool okr = colok && zr >= 0 && zr < g.Nz;
    const long long cr = okr ? (long long)zr * pitch + xc : 0;
    const bool okk = colok && k >= 0 && k < g.Nz;
    const long long ck = okk ? (long long)k * pitch + xc : 0;
    // free surface: the pressure pair of a ghost row and v_z of a ghost half
    // row come from their mirror rows
    bool okrs = okr, okks = okk;
    long long crs = cr, cks = ck;
    if constexpr (FS) {
        const int zrs = node_src_row<FS>(g, zr), ks = half_src_row<FS>(g, k);
        okrs = colok && zrs >= 0 && zrs < g.Nz;
        crs = okrs ? (long long)zrs * pitch + xc : 0;
        okks = okk && ks < g.Nz;
        cks = okks ? (long long)ks * pitch + xc : 0;
    }
    const bool okk1 = colok && k + 1 >= 0;
    const long long ck1 = okk1 ? (long long)min(k + 1, g.Nz - 1) * pitch + xc : 0;
    const bool main = z >= zc0 && z < zc1;
    const bool okz = colok && main;
    const long long cz = okz ? (long long)z * pitch + xc : 0;
    const bool okv = vxok && main;
    const int iz = z - z0;
    cpa(s2 + 0 * NTH, in2 + (A_PL / 2) * p2 + crs, okrs);
    cpa(s2 + 1 * NTH, in2 + (A_VZ / 2) * p2 + cks, okks);
    cpa(s2 + 2 * NTH, in2 + (A_PL / 2) * p2 + cz, okz);
    cpa(s2 + 3 * NTH, in2 + (A_VX / 2) * p2 + cz, okv);
    cpa(s2 + 4 * NTH, img + cz, outcol && main && inner_col && iz >= 0 && iz < g.nz);
    const float *kdt = WIN ? in + W_KDT * plane : a.kdt;
    const float *binv = WIN ? in + W_BINV * plane : a.binv;
    cpa(s1 + 0 * NTH, kdt + cr, okr);
    cpa(s1 + 1 * NTH, in + A_LPVZ * plane + cr, okr && ((zr <= z0 - 1) || (zr >= z1)));
    cpa(s1 + 2 * NTH, binv + ck1, okk1);
    cpa(s1 + 3 * NTH, in + A_LPPZ * plane + ck, okk && ((k <= z0 - 2) || (k >= z1)));
    cpa(s1 + 4 * NTH, kdt + cz, okz);
    cpa(s1 + 5 * NTH, in + A_LPVX * plane + cz, okz && pmlxn);
    cpa(s1 + 6 * NTH, in + A_LPVZ * plane + cz, outcol && main && ((z <= z0 - 1) || (z >= z1)));
    cpa(s1 + 7 * NTH, binv + cz, okz);
    cpa(s1 + 8 * NTH, in + A_LPPX * plane + cz, okv && pmlxh);
}

__device__ __forceinline__ AdjRow adj_read(const float *st)
{
    const int t = threadIdx.x;
    const float2 *s2 = reinterpret_cast<const float2 *>(st) + t;
    const float *s1 = st + 2 * kAdjF2 * NTH + t;
    AdjRow r;
    r.pl = s2[0 * NTH];
    r.v2z = s2[1 * NTH];
    r.plz = s2[2 * NTH];
    r.v2x = s2[3 * NTH];
    r.img = s2[4 * NTH];
    r.kdr = s1[0 * NTH];
    r.lpvzr = s1[1 * NTH];
    r.bz = s1[2 * NTH];
    r.lppz = s1[3 * NTH];
    r.kdz = s1[4 * NTH];
    r.lpsvx = s1[5 * NTH];
    r.lpsvz = s1[6 * NTH];
    r.bx = s1[7 * NTH];
    r.lppx = s1[8 * NTH];
    return r;
}

template <int M, bool WIN, bool FS>
__global__ void __launch_bounds__(NTH, FS ? kAdjMinBlocksFS : kAdjMinBlocks) k_adj2d(const Step2D a)
{
    if (guard_tripped(a.g)) return;
    using C = Cols<M>;
    constexpr int W = C::W, HXP = C::HXP, TXO = C::TXO;
    __shared__ float2 sPU[NTH];   // (p^n, kdt*lp - ai_x (lpsi_vx - kdt*lp)), row z
    __shared__ float sB[NTH];     // 1/rho, row z
    __shared__ float2 sVW[NTH];   // (vx^{n+1/2}, dt*bu_x*lvx - ah_x*lpsi_px), row z
    __shared__ float sVN[NTH];    // vx^{n-1/2}, row z
    __shared__ float sPi[NTH];    // Gx * lvx, row z
    extern __shared__ __align__(16) float stagef[];   // [PDA][kAdjStageFloats]

    const GridDev &g = a.g;
    const int t = threadIdx.x;
    const int slot = blockIdx.z, shot = a.shot0 + slot;
    // padded and interior widths of this shot's grid (its aperture window)
    const int Nx = WIN ? a.win_nx[shot] + 2 * g.x0 : g.Nx;
    const int nx = WIN ? Nx - 2 * g.x0 : g.nx;
    if (WIN && (int)blockIdx.x * TXO >= Nx) return;   // no output column in this shot's window
    const int x = (int)blockIdx.x * TXO - HXP + t;
    const bool colok = x >= 0 && x < Nx;
    const bool outcol = colok && t >= HXP && t < HXP + TXO;
    const bool vxok = colok && t >= M - 1 && t <= NTH - 1 - M;
    const int zc0 = (int)blockIdx.y * a.tzc;
    const int zc1 = min(zc0 + a.tzc, g.Nz);
    const int zstart = zc0 - W;
    const long long plane = g.plane;
    const long long p2 = plane;   // stride of one pair field in float2 units
    const int pitch = g.pitch;
    const int xc = colok ? x : 0;
    const float *in = a.in + slot * a.sstride;
    float *outf = a.out + slot * a.sstride + xc;
    float2 *out2 = reinterpret_cast<float2 *>(a.out + slot * a.sstride) + xc;
    const float dt = g.dt;
    const int n = a.n;
    const bool recon = n > 0;
    const int x0 = g.x0, x1 = g.x0 + nx, z0 = g.z0, z1 = g.z0 + g.nz;
    const int ix = x - x0;
    const bool xint = ix >= 0 && ix < nx;
    const bool pmlxh = colok && ((x <= x0 - 2) || (x >= x1));
    const bool pmlxn = colok && ((x <= x0 - 1) || (x >= x1));
    const int px = WIN ? shot * a.pml_xstride + x : x;   // x CPML profiles of this shot's window
    const float ahx = pmlxh ? a.pml.ah[2][px] : 0.f, bhx = pmlxh ? a.pml.bh[2][px] : 0.f;
    const float aix = pmlxn ? a.pml.ai[2][px] : 0.f, bix = pmlxn ? a.pml.bi[2][px] : 0.f;
    const long long rowprev = band_row(a.bands, shot, n - 1);
    const int src = a.src_cell[shot];
    const float wsrc = recon ? a.src_scale * a.wav[(a.wav_per_shot ? (long long)shot * g.nt : 0) + n - 1] : 0.f;
    const float2 *imgs = a.img + slot * plane;   // image accumulators of this slot
    float2 *img = a.img + slot * plane + xc;

    // z rings, shifted by U entries after every group of U rows: at row u of a
    // group, entry u + m holds node row z + m (PU) or the half-row value
    // written m - W + 1 rows earlier (VW, VN, PIZ), m = 0 .. W - 1
    constexpr int U = W / kAdjGroupDiv > 0 ? W / kAdjGroupDiv : 1, RL = W + U - 1;
    float2 PU[RL], VW[RL];
    float VN[RL], PIZ[RL];
#pragma unroll
    for (int j = 0; j < RL; ++j) {
        PU[j] = make_float2(0.f, 0.f);
        VW[j] = make_float2(0.f, 0.f);
        VN[j] = 0.f;
        PIZ[j] = 0.f;
    }
    // (p^n, kdt*lp - ai_z (lpsi_vz - kdt*lp)) at node row r of this column
    // (pl holds the mirror row's values for a ghost row r < z0; the surface
    // row carries p = 0 and lambda_p = 0)
    auto pu_node = [&](int r, float2 pl, float kd, float lpvz) -> float2 {
        if (FS && r <= z0) {
            if (r == z0) return make_float2(0.f, 0.f);
            return make_float2(-pl.x, -(kd * pl.y));
        }
        float kl = kd * pl.y;
        if (colok && r >= 0 && r < g.Nz && ((r <= z0 - 1) || (r >= z1))) kl -= a.pml.ai[0][r] * (lpvz - kl);
        return make_float2(pl.x, kl);
    };
    {
        const float2 *in2 = reinterpret_cast<const float2 *>(in);
#pragma unroll
        for (int j = 0; j < W - 1; ++j) {
            const int r = zstart + j, rs = node_src_row<FS>(g, r);
            const bool ok = colok && r >= 0 && r < g.Nz;
            const long long cr = ok ? (long long)r * pitch + xc : 0;
            const bool oks = colok && rs >= 0 && rs < g.Nz;
            const float2 plv = oks ? in2[(A_PL / 2) * p2 + (long long)rs * pitch + xc] : make_float2(0.f, 0.f);
            const float kd = ok ? (WIN ? in[W_KDT * plane + cr] : a.kdt[cr]) : 0.f;
            const float lpvz = (ok && ((r <= z0 - 1) || (r >= z1))) ? in[A_LPVZ * plane + cr] : 0.f;
            PU[j] = pu_node(r, plv, kd, lpvz);
        }
    }
    float bz_old = 0.f;
    {
        int k = zstart + M - 1;
        if (colok && k >= 0 && k < g.Nz)
            bz_old = WIN ? in[W_BINV * plane + (long long)k * pitch + xc] : a.binv[(long long)k * pitch + xc];
    }

#pragma unroll
    for (int j = 0; j < PDA - 1; ++j) {
        if (zstart + j < zc1)
            adj_issue<M, WIN, FS>(stagef + j * kAdjStageFloats, a, imgs, in, xc, zstart + j, zc0, zc1, colok, vxok,
                         outcol, pmlxh, pmlxn, xint);
        cp_commit();
    }

    for (int zb = zstart; zb < zc1; zb += U) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int z = zb + u;
            if (z >= zc1) break;
            const int zi = z + PDA - 1;
            if (zi < zc1)
                adj_issue<M, WIN, FS>(stagef + ((zi - zstart) % PDA) * kAdjStageFloats, a, imgs, in, xc, zi, zc0, zc1,
                             colok, vxok, outcol, pmlxh, pmlxn, xint);
            cp_commit();
            cp_wait_row<PDA>();
            const AdjRow cur = adj_read(stagef + ((z - zstart) % PDA) * kAdjStageFloats);
            const int k = z + M - 1;
            const int sl = u + W - 1;
            PU[sl] = pu_node(z + W - 1, cur.pl, cur.kdr, cur.lpvzr);
            const float buz = 0.5f * (bz_old + cur.bz);
            bz_old = cur.bz;
            // ---- half row k along z: lambda_vz, lambda_psi_pz, background vz^{n-1/2}
            float wz = 0.f, vn = 0.f, piz = 0.f;
            if (colok && k >= 0 && k < g.Nz) {
                const long long ck = (long long)k * pitch;
                const bool own = outcol && k >= zc0 && k < zc1;
                // (Gz, du/dz)
                const float2 D = stencil<M, float2>(g.cz, [&](int l) { return PU[u + M - 1 + l]; },
                                                    [&](int l) { return PU[u + M - l]; });
                const float lv = cur.v2z.y + D.y;
                const float dtbu = dt * buz;
                wz = dtbu * lv;
                if ((k <= z0 - 2) || (k >= z1)) {
                    float l1 = cur.lppz - dtbu * lv;
                    wz -= a.pml.ah[0][k] * l1;
                    if (own) outf[A_LPPZ * plane + ck] = a.pml.bh[0][k] * l1;
                }
                piz = D.x * lv;
                if (recon && xint) {
                    const int iz = k - z0;
                    if ((iz >= 0 || FS) && iz < g.nz) vn = cur.v2z.x + dtbu * D.x;
                    else if (in_xstrip(iz, M, g.nz))
                        vn = band_get(a.bands, 1, rowprev, band_zstrip(iz, ix, M, g.nz, nx));
                }
                if (own) out2[(A_VZ / 2) * p2 + ck] = make_float2(vn, lv);
            }
            VW[sl] = make_float2(cur.v2z.x, wz);
            VN[sl] = vn;
            PIZ[sl] = piz;
            if (z < zc0) continue;

            // ---- row z: half nodes along x
            const long long cz = (long long)z * pitch;
            const bool surf = FS && z == z0;   // free-surface row: p = 0, lambda_p = 0
            const float pbn = cur.plz.x;
            const float lp1 = surf ? 0.f : cur.plz.y;
            const float kd = cur.kdz;
            const float kl = kd * lp1;
            sPU[t] = make_float2(pbn, pmlxn ? kl - aix * (cur.lpsvx - kl) : kl);
            sB[t] = cur.bx;
            __syncthreads();
            float2 vw = make_float2(cur.v2x.x, 0.f);
            float vxn = 0.f, pix = 0.f;
            if (vxok) {
                // (Gx, du/dx)
                const float2 D = stencil<M, float2>(g.cx, [&](int l) { return sPU[t + l]; },
                                                    [&](int l) { return sPU[t + 1 - l]; });
                const float bux = 0.5f * (cur.bx + (x + 1 >= Nx ? cur.bx : sB[t + 1]));
                const float dtbu = dt * bux;
                const float lv = cur.v2x.y + D.y;
                float wx = dtbu * lv;
                if (pmlxh) {
                    float l1 = cur.lppx - dtbu * lv;
                    wx -= ahx * l1;
                    if (outcol) outf[A_LPPX * plane + cz] = bhx * l1;
                }
                vw.y = wx;
                pix = D.x * lv;
                if (recon) {
                    const int iz = z - z0;
                    if (iz >= 0 && iz < g.nz) {
                        if (xint) vxn = cur.v2x.x + dtbu * D.x;
                        else if (in_xstrip(ix, M, nx))
                            vxn = band_get(a.bands, 1, rowprev, band_xstrip(iz, ix, M, g.nz, nx));
                    }
                }
                if (outcol) out2[(A_VX / 2) * p2 + cz] = make_float2(vxn, lv);
            }
            sVW[t] = vw;
            sVN[t] = vxn;
            sPi[t] = pix;
            __syncthreads();

            // ---- row z: nodes on the output columns
            if (outcol) {
                // (Q_n, D- w) along x and z
                const float2 Ex = stencil<M, float2>(g.cx, [&](int l) { return sVW[t + l - 1]; },
                                                     [&](int l) { return sVW[t - l]; });
                const float2 Ez = stencil<M, float2>(g.cz, [&](int l) { return VW[u + M + l - 1]; },
                                                     [&](int l) { return VW[u + M - l]; });
                const float2 E = add_(Ex, Ez);
                float qn = 0.f;
                if (recon)
                    qn = stencil<M, float>(g.cx, [&](int l) { return sVN[t + l - 1]; }, [&](int l) { return sVN[t - l]; }) +
                         stencil<M, float>(g.cz, [&](int l) { return VN[u + M + l - 1]; },
                                           [&](int l) { return VN[u + M - l]; });
                const int iz = z - z0;
                const bool inner = xint && iz >= 0 && iz < g.nz;
                if (inner) {
                    float2 acc = cur.img;
                    acc.x += E.x * lp1;
                    // (on the free surface the half row above is a ghost: no product of its own)
                    acc.y += (sPi[t] + sPi[t - 1]) + (PIZ[u + M] + (surf ? 0.f : PIZ[u + M - 1]));
                    img[cz] = acc;
                }
                float pn = 0.f;
                if (recon) {
                    if (inner) {
                        pn = pbn + kd * qn;
                        if (cz + x == src) pn -= wsrc;
                    } else {
                        long long b = pband_index(iz, ix, M, g.nz, nx);
                        if (b >= 0) pn = band_get(a.bands, 0, rowprev, b);
                    }
                }
                out2[(A_PL / 2) * p2 + cz] = (FS && z <= z0) ? make_float2(0.f, 0.f) : make_float2(pn, lp1 + E.y);
                if (pmlxn) outf[A_LPVX * plane + cz] = bix * (cur.lpsvx - kl);
                if ((z <= z0 - 1) || (z >= z1)) outf[A_LPVZ * plane + cz] = a.pml.bi[0][z] * (cur.lpsvz - kl);
            }
        }
#pragma unroll
        for (int j = 0; j < W - 1; ++j) {
            PU[j] = PU[j + U];
            VW[j] = VW[j + U];
            VN[j] = VN[j + U];
            PIZ[j] = PIZ[j + U];
        }
    }

    if (recon) {
        // pre-add the residual of step n-1 at the receivers of this CTA
        __syncthreads();
        int tile = shot * a.trec.ntiles + blockIdx.y * gridDim.x + blockIdx.x;
        int b = a.trec.ptr[tile], e = a.trec.ptr[tile + 1];
        float2 *plo = reinterpret_cast<float2 *>(a.out + slot * a.sstride + A_PL * plane);
        for (int i = b + t; i < e; i += NTH) {
            int2 rc = a.trec.rec[i];
            if (i > b && a.trec.rec[i - 1].x == rc.x) continue;  // run handled by its first entry
            float add = 0.f;
            for (int q = i; q < e && a.trec.rec[q].x == rc.x; ++q)
                add += a.dstage[(long long)a.trec.rec[q].y * g.nt + (n - 1)];
            plo[rc.x].y += add;
        }
    }
}

// Start state of a reverse pass: (p, 0), (vx, 0), (vz, 0) from the saved
// background final state [p][vx][vz] of each shot of the batch.
// ---------------------------------------------------------------------------
// Migration step with TMA row staging (shots without aperture windows). The
// same arithmetic as k_adj2d, in the same order, so the results are the same
// bits; only the loads of the rows ahead differ. One thread (the last) issues
// every field row of a stage as one tensor-map tile copy (a kThreads2D-wide
// row of one field) on the stage's mbarrier; the tensor maps read zeros
// outside the padded grid, which is what the per-thread copies' zero fill
// gives at the grid edges. Rows the per-thread copies zero-fill inside the
// grid (a row whose source row is out of range) are read from row -1.
// Fields a row does not use (the CPML memories outside the strips, the
// row-z fields of the warm-up rows) are not copied; no consumer reads them.
// A stage is refilled only after a CTA barrier that follows every read of
// it: the previous row's barriers (a warm-up row adds one for this).
// ---------------------------------------------------------------------------
struct Adj2T {
    Step2D a;
    Maps2D m;
};

constexpr unsigned kAdjStageBytesT = (unsigned)(kAdjStageFloats * sizeof(float));
static_assert(kAdjStageBytesT % 128 == 0, "stage rows stay 128-byte aligned");
constexpr unsigned kAdjBarOff = PDA * kAdjStageBytesT;
constexpr unsigned kAdjSmemT = kAdjBarOff + 64 + 128;   // stages, barriers, alignment slack

// Issues the copies of row z (the stage layout of adj_issue) on barrier b.
// xs: first column of the CTA (a multiple of 4, so every copy starts on a
// 16-byte boundary); tpn / tph: the CTA has node / half-node CPML columns.
template <int M, bool FS>
__device__ __forceinline__ void adj_issue_tma(const Adj2T &p, float *st, uint64_t *b, int slot, int xs, int z,
                                              int zc0, int zc1, bool tpn, bool tph)
{
    const GridDev &g = p.a.g;
    const Maps2D &m = p.m;
    constexpr int W = 2 * M;
    constexpr unsigned R2 = NTH * 8, R1 = NTH * 4;   // bytes of one float2 / float field row
    const int z0 = g.z0, z1 = g.z0 + g.nz;
    const int zr = z + W - 1, k = z + M - 1;
    const int qp = slot * m.pps, qf = slot * m.fps;
    char *s2 = reinterpret_cast<char *>(st);
    char *s1 = s2 + kAdjF2 * R2;
    const bool inr = zr >= 0 && zr < g.Nz, ink = k >= 0 && k < g.Nz;
    int rpl = zr, rvz = ink ? k : -1;
    if constexpr (FS) {
        const int zrs = node_src_row<FS>(g, zr), ks = half_src_row<FS>(g, k);
        rpl = (zrs >= 0 && zrs < g.Nz) ? zrs : -1;
        rvz = (ink && ks < g.Nz) ? ks : -1;
    }
    const int rbz = k + 1 >= 0 ? min(k + 1, g.Nz - 1) : -1;
    const bool lpa = inr && ((zr <= z0 - 1) || (zr >= z1));
    const bool lpz = ink && ((k <= z0 - 2) || (k >= z1));
    const bool main = z >= zc0 && z < zc1;
    const int iz = z - z0;
    const bool im = main && iz >= 0 && iz < g.nz;
    const bool lvx = main && tpn, lvz = main && ((z <= z0 - 1) || (z >= z1)), lpx = main && tph;
    unsigned bytes = 2 * R2 + 2 * R1 + (lpa ? R1 : 0) + (lpz ? R1 : 0);
    if (main) bytes += 2 * R2 + 2 * R1;
    if (im) bytes += R2;
    if (lvx) bytes += R1;
    if (lvz) bytes += R1;
    if (lpx) bytes += R1;
    tma::fence_proxy_async();
    tma::mbar_expect(b, bytes);
    tma::load3(s2 + 0 * R2, m.pr, xs, rpl, qp + A_PL / 2, b);
    tma::load3(s2 + 1 * R2, m.pr, xs, rvz, qp + A_VZ / 2, b);
    tma::load3(s1 + 0 * R1, m.md, xs, zr, 0, b);
    if (lpa) tma::load3(s1 + 1 * R1, m.fl, xs, zr, qf + A_LPVZ, b);
    tma::load3(s1 + 2 * R1, m.md, xs, rbz, 1, b);
    if (lpz) tma::load3(s1 + 3 * R1, m.fl, xs, k, qf + A_LPPZ, b);
    if (main) {
        tma::load3(s2 + 2 * R2, m.pr, xs, z, qp + A_PL / 2, b);
        tma::load3(s2 + 3 * R2, m.pr, xs, z, qp + A_VX / 2, b);
        tma::load3(s1 + 4 * R1, m.md, xs, z, 0, b);
        tma::load3(s1 + 7 * R1, m.md, xs, z, 1, b);
    }
    if (im) tma::load3(s2 + 4 * R2, m.im, xs, z, slot, b);
    if (lvx) tma::load3(s1 + 5 * R1, m.fl, xs, z, qf + A_LPVX, b);
    if (lvz) tma::load3(s1 + 6 * R1, m.fl, xs, z, qf + A_LPVZ, b);
    if (lpx) tma::load3(s1 + 8 * R1, m.fl, xs, z, qf + A_LPPX, b);
}

template <int M, bool FS>
__global__ void __launch_bounds__(NTH, FS ? kAdjMinBlocksFS : kAdjMinBlocks) k_adj2t(const __grid_constant__ Adj2T p)
{
    const Step2D &a = p.a;
    if (guard_tripped(a.g)) return;
    using C = Cols<M>;
    constexpr int W = C::W, HXP = C::HXP, TXO = C::TXO;
    static_assert(TXO % 4 == 0 && HXP % 4 == 0, "CTA column starts must be 16-byte aligned for 4-byte elements");
    __shared__ float2 sPU[NTH];   // (p^n, kdt*lp - ai_x (lpsi_vx - kdt*lp)), row z
    __shared__ float sB[NTH];     // 1/rho, row z
    __shared__ float2 sVW[NTH];   // (vx^{n+1/2}, dt*bu_x*lvx - ah_x*lpsi_px), row z
    __shared__ float sVN[NTH];    // vx^{n-1/2}, row z
    __shared__ float sPi[NTH];    // Gx * lvx, row z
    extern __shared__ unsigned char smraw[];
    unsigned char *sm = smraw + ((128u - (tma::su32(smraw) & 127u)) & 127u);
    float *stagef = reinterpret_cast<float *>(sm);   // [PDA][kAdjStageFloats]
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kAdjBarOff);

    const GridDev &g = a.g;
    const int t = threadIdx.x;
    const int slot = blockIdx.z, shot = a.shot0 + slot;
    const int Nx = g.Nx, nx = g.nx;
    const int xs = (int)blockIdx.x * TXO - HXP;
    const int x = xs + t;
    const bool colok = x >= 0 && x < Nx;
    const bool outcol = colok && t >= HXP && t < HXP + TXO;
    const bool vxok = colok && t >= M - 1 && t <= NTH - 1 - M;
    const int zc0 = (int)blockIdx.y * a.tzc;
    const int zc1 = min(zc0 + a.tzc, g.Nz);
    const int zstart = zc0 - W;
    const long long plane = g.plane;
    const long long p2 = plane;   // stride of one pair field in float2 units
    const int pitch = g.pitch;
    const int xc = colok ? x : 0;
    const float *in = a.in + slot * a.sstride;
    float *outf = a.out + slot * a.sstride + xc;
    float2 *out2 = reinterpret_cast<float2 *>(a.out + slot * a.sstride) + xc;
    const float dt = g.dt;
    const int n = a.n;
    const bool recon = n > 0;
    const int x0 = g.x0, x1 = g.x0 + nx, z0 = g.z0, z1 = g.z0 + g.nz;
    const int ix = x - x0;
    const bool xint = ix >= 0 && ix < nx;
    const bool pmlxh = colok && ((x <= x0 - 2) || (x >= x1));
    const bool pmlxn = colok && ((x <= x0 - 1) || (x >= x1));
    const bool tph = (xs <= x0 - 2) || (xs + NTH - 1 >= x1);   // CTA has half-node / node CPML columns
    const bool tpn = (xs <= x0 - 1) || (xs + NTH - 1 >= x1);
    const float ahx = pmlxh ? a.pml.ah[2][x] : 0.f, bhx = pmlxh ? a.pml.bh[2][x] : 0.f;
    const float aix = pmlxn ? a.pml.ai[2][x] : 0.f, bix = pmlxn ? a.pml.bi[2][x] : 0.f;
    const long long rowprev = band_row(a.bands, shot, n - 1);
    const int src = a.src_cell[shot];
    const float wsrc = recon ? a.src_scale * a.wav[(a.wav_per_shot ? (long long)shot * g.nt : 0) + n - 1] : 0.f;
    float2 *img = a.img + slot * plane + xc;
    constexpr int PR = NTH - 1;   // the thread that issues the copies

    if (t == 0) {
        for (int i = 0; i < PDA; ++i) tma::mbar_init(bar + i);
        tma::mbar_init_fence();
    }
    __syncthreads();
    if (t == PR) {
        for (int j = 0; j < PDA - 1 && zstart + j < zc1; ++j)
            adj_issue_tma<M, FS>(p, stagef + j * kAdjStageFloats, bar + j, slot, xs, zstart + j, zc0, zc1, tpn, tph);
    }

    constexpr int U = W / kAdjGroupDiv > 0 ? W / kAdjGroupDiv : 1, RL = W + U - 1;
    float2 PU[RL], VW[RL];
    float VN[RL], PIZ[RL];
#pragma unroll
    for (int j = 0; j < RL; ++j) {
        PU[j] = make_float2(0.f, 0.f);
        VW[j] = make_float2(0.f, 0.f);
        VN[j] = 0.f;
        PIZ[j] = 0.f;
    }
    auto pu_node = [&](int r, float2 pl, float kd, float lpvz) -> float2 {
        if (FS && r <= z0) {
            if (r == z0) return make_float2(0.f, 0.f);
            return make_float2(-pl.x, -(kd * pl.y));
        }
        float kl = kd * pl.y;
        if (colok && r >= 0 && r < g.Nz && ((r <= z0 - 1) || (r >= z1))) kl -= a.pml.ai[0][r] * (lpvz - kl);
        return make_float2(pl.x, kl);
    };
    {
        const float2 *in2 = reinterpret_cast<const float2 *>(in);
#pragma unroll
        for (int j = 0; j < W - 1; ++j) {
            const int r = zstart + j, rs = node_src_row<FS>(g, r);
            const bool ok = colok && r >= 0 && r < g.Nz;
            const long long cr = ok ? (long long)r * pitch + xc : 0;
            const bool oks = colok && rs >= 0 && rs < g.Nz;
            const float2 plv = oks ? in2[(A_PL / 2) * p2 + (long long)rs * pitch + xc] : make_float2(0.f, 0.f);
            const float kd = ok ? a.kdt[cr] : 0.f;
            const float lpvz = (ok && ((r <= z0 - 1) || (r >= z1))) ? in[A_LPVZ * plane + cr] : 0.f;
            PU[j] = pu_node(r, plv, kd, lpvz);
        }
    }
    float bz_old = 0.f;
    {
        int k = zstart + M - 1;
        if (colok && k >= 0 && k < g.Nz) bz_old = a.binv[(long long)k * pitch + xc];
    }

    bool bad = false;      // this thread's wait gave up
    int fail_row = zc1;    // first row whose stage was not consumed
    for (int zb = zstart; zb < zc1; zb += U) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int z = zb + u;
            if (z >= zc1) break;
            const int j = z - zstart;
            // refill the stage of row z - 1 with row z + PDA - 1: every thread
            // passed a barrier after reading it (the previous row's)
            const int zi = z + PDA - 1;
            if (t == PR && zi < zc1)
                adj_issue_tma<M, FS>(p, stagef + ((j + PDA - 1) % PDA) * kAdjStageFloats, bar + (j + PDA - 1) % PDA,
                                     slot, xs, zi, zc0, zc1, tpn, tph);
            bad |= !tma::mbar_wait(bar + j % PDA, (unsigned)(j / PDA) & 1u);
            const AdjRow cur = adj_read(stagef + (j % PDA) * kAdjStageFloats);
            const int k = z + M - 1;
            const int sl = u + W - 1;
            PU[sl] = pu_node(z + W - 1, cur.pl, cur.kdr, cur.lpvzr);
            const float buz = 0.5f * (bz_old + cur.bz);
            bz_old = cur.bz;
            // ---- half row k along z: lambda_vz, lambda_psi_pz, background vz^{n-1/2}
            float wz = 0.f, vn = 0.f, piz = 0.f;
            if (colok && k >= 0 && k < g.Nz) {
                const long long ck = (long long)k * pitch;
                const bool own = outcol && k >= zc0 && k < zc1;
                const float2 D = stencil<M, float2>(g.cz, [&](int l) { return PU[u + M - 1 + l]; },
                                                    [&](int l) { return PU[u + M - l]; });
                const float lv = cur.v2z.y + D.y;
                const float dtbu = dt * buz;
                wz = dtbu * lv;
                if ((k <= z0 - 2) || (k >= z1)) {
                    float l1 = cur.lppz - dtbu * lv;
                    wz -= a.pml.ah[0][k] * l1;
                    if (own) outf[A_LPPZ * plane + ck] = a.pml.bh[0][k] * l1;
                }
                piz = D.x * lv;
                if (recon && xint) {
                    const int iz = k - z0;
                    if ((iz >= 0 || FS) && iz < g.nz) vn = cur.v2z.x + dtbu * D.x;
                    else if (in_xstrip(iz, M, g.nz))
                        vn = band_get(a.bands, 1, rowprev, band_zstrip(iz, ix, M, g.nz, nx));
                }
                if (own) out2[(A_VZ / 2) * p2 + ck] = make_float2(vn, lv);
            }
            VW[sl] = make_float2(cur.v2z.x, wz);
            VN[sl] = vn;
            PIZ[sl] = piz;
            if (z < zc0) {
                // warm-up row: the barrier that lets its stage be refilled
                if (__syncthreads_or(bad)) {
                    fail_row = z;
                    break;
                }
                continue;
            }

            // ---- row z: half nodes along x
            const long long cz = (long long)z * pitch;
            const bool surf = FS && z == z0;   // free-surface row: p = 0, lambda_p = 0
            const float pbn = cur.plz.x;
            const float lp1 = surf ? 0.f : cur.plz.y;
            const float kd = cur.kdz;
            const float kl = kd * lp1;
            sPU[t] = make_float2(pbn, pmlxn ? kl - aix * (cur.lpsvx - kl) : kl);
            sB[t] = cur.bx;
            if (__syncthreads_or(bad)) {
                fail_row = z;
                break;
            }
            float2 vw = make_float2(cur.v2x.x, 0.f);
            float vxn = 0.f, pix = 0.f;
            if (vxok) {
                const float2 D = stencil<M, float2>(g.cx, [&](int l) { return sPU[t + l]; },
                                                    [&](int l) { return sPU[t + 1 - l]; });
                const float bux = 0.5f * (cur.bx + (x + 1 >= Nx ? cur.bx : sB[t + 1]));
                const float dtbu = dt * bux;
                const float lv = cur.v2x.y + D.y;
                float wx = dtbu * lv;
                if (pmlxh) {
                    float l1 = cur.lppx - dtbu * lv;
                    wx -= ahx * l1;
                    if (outcol) outf[A_LPPX * plane + cz] = bhx * l1;
                }
                vw.y = wx;
                pix = D.x * lv;
                if (recon) {
                    const int iz = z - z0;
                    if (iz >= 0 && iz < g.nz) {
                        if (xint) vxn = cur.v2x.x + dtbu * D.x;
                        else if (in_xstrip(ix, M, nx))
                            vxn = band_get(a.bands, 1, rowprev, band_xstrip(iz, ix, M, g.nz, nx));
                    }
                }
                if (outcol) out2[(A_VX / 2) * p2 + cz] = make_float2(vxn, lv);
            }
            sVW[t] = vw;
            sVN[t] = vxn;
            sPi[t] = pix;
            __syncthreads();

            // ---- row z: nodes on the output columns
            if (outcol) {
                const float2 Ex = stencil<M, float2>(g.cx, [&](int l) { return sVW[t + l - 1]; },
                                                     [&](int l) { return sVW[t - l]; });
                const float2 Ez = stencil<M, float2>(g.cz, [&](int l) { return VW[u + M + l - 1]; },
                                                     [&](int l) { return VW[u + M - l]; });
                const float2 E = add_(Ex, Ez);
                float qn = 0.f;
                if (recon)
                    qn = stencil<M, float>(g.cx, [&](int l) { return sVN[t + l - 1]; }, [&](int l) { return sVN[t - l]; }) +
                         stencil<M, float>(g.cz, [&](int l) { return VN[u + M + l - 1]; },
                                           [&](int l) { return VN[u + M - l]; });
                const int iz = z - z0;
                const bool inner = xint && iz >= 0 && iz < g.nz;
                if (inner) {
                    float2 acc = cur.img;
                    acc.x += E.x * lp1;
                    // (on the free surface the half row above is a ghost: no product of its own)
                    acc.y += (sPi[t] + sPi[t - 1]) + (PIZ[u + M] + (surf ? 0.f : PIZ[u + M - 1]));
                    img[cz] = acc;
                }
                float pn = 0.f;
                if (recon) {
                    if (inner) {
                        pn = pbn + kd * qn;
                        if (cz + x == src) pn -= wsrc;
                    } else {
                        long long b = pband_index(iz, ix, M, g.nz, nx);
                        if (b >= 0) pn = band_get(a.bands, 0, rowprev, b);
                    }
                }
                out2[(A_PL / 2) * p2 + cz] = (FS && z <= z0) ? make_float2(0.f, 0.f) : make_float2(pn, lp1 + E.y);
                if (pmlxn) outf[A_LPVX * plane + cz] = bix * (cur.lpsvx - kl);
                if ((z <= z0 - 1) || (z >= z1)) outf[A_LPVZ * plane + cz] = a.pml.bi[0][z] * (cur.lpsvz - kl);
            }
        }
        if (fail_row < zc1) break;
#pragma unroll
        for (int j = 0; j < W - 1; ++j) {
            PU[j] = PU[j + U];
            VW[j] = VW[j + U];
            VN[j] = VN[j + U];
            PIZ[j] = PIZ[j + U];
        }
    }

    if (fail_row < zc1) {
        // a wait gave up: record it, let the copies in flight land (rows up to
        // fail_row + PDA - 1 were issued), return
        if (t == PR) {
            atomicOr(a.err, 1);
            for (int zz = fail_row; zz <= min(fail_row + PDA - 1, zc1 - 1); ++zz) {
                const int jj = zz - zstart;
                (void)tma::mbar_wait(bar + jj % PDA, (unsigned)(jj / PDA) & 1u);
            }
        }
        return;
    }

    if (recon) {
        // pre-add the residual of step n-1 at the receivers of this CTA
        __syncthreads();
        int tile = shot * a.trec.ntiles + blockIdx.y * gridDim.x + blockIdx.x;
        int b = a.trec.ptr[tile], e = a.trec.ptr[tile + 1];
        float2 *plo = reinterpret_cast<float2 *>(a.out + slot * a.sstride + A_PL * plane);
        for (int i = b + t; i < e; i += NTH) {
            int2 rc = a.trec.rec[i];
            if (i > b && a.trec.rec[i - 1].x == rc.x) continue;  // run handled by its first entry
            float add = 0.f;
            for (int q = i; q < e && a.trec.rec[q].x == rc.x; ++q)
                add += a.dstage[(long long)a.trec.rec[q].y * g.nt + (n - 1)];
            plo[rc.x].y += add;
        }
    }
}

__global__ void k_pack_adj(const GridDev g, const float *final_state, int shot0, int batch, float *st,
                           long long sstride)
{
    const long long plane = g.plane;
    const long long n = batch * plane;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long s = i / plane, c = i - s * plane;
        const float *fs = final_state + (shot0 + s) * 3 * plane;
        float2 *o = reinterpret_cast<float2 *>(st + s * sstride);
        o[(A_PL / 2) * plane + c] = make_float2(fs[c], 0.f);
        o[(A_VX / 2) * plane + c] = make_float2(fs[plane + c], 0.f);
        o[(A_VZ / 2) * plane + c] = make_float2(fs[2 * plane + c], 0.f);
    }
}

template <int M, bool BORN, bool BANDS, bool HESS, bool WIN>
cudaError_t launch_fwd_t(const Step2D &a, dim3 grid, cudaStream_t s)
{
    if (a.g.fs) k_fwd2d<M, BORN, BANDS, HESS, WIN, true><<<grid, NTH, kFwdStageBytes, s>>>(a);
    else k_fwd2d<M, BORN, BANDS, HESS, WIN, false><<<grid, NTH, kFwdStageBytes, s>>>(a);
    return cudaGetLastError();
}

template <int M, bool BORN, bool BANDS, bool HESS>
cudaError_t attr_fwd()
{
    cudaError_t e;
    const int b = (int)kFwdStageBytes;
    const auto at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(k_fwd2d<M, BORN, BANDS, HESS, false, false>, at, b)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_fwd2d<M, BORN, BANDS, HESS, true, false>, at, b)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_fwd2d<M, BORN, BANDS, HESS, false, true>, at, b)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_fwd2d<M, BORN, BANDS, HESS, true, true>, at, b);
}

template <int M>
cudaError_t attr_M()
{
    cudaError_t e;
    if ((e = attr_fwd<M, true, false, false>()) != cudaSuccess) return e;
    if ((e = attr_fwd<M, false, true, true>()) != cudaSuccess) return e;
    if ((e = attr_fwd<M, false, true, false>()) != cudaSuccess) return e;
    if ((e = attr_fwd<M, false, false, true>()) != cudaSuccess) return e;
    if ((e = attr_fwd<M, false, false, false>()) != cudaSuccess) return e;
    const int b = (int)kAdjStageBytes;
    const auto at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(k_adj2d<M, false, false>, at, b)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_adj2d<M, true, false>, at, b)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_adj2d<M, false, true>, at, b)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_adj2d<M, true, true>, at, b)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_fwd2t<M, false>, at, (int)kFwdSmemT)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_fwd2t<M, true>, at, (int)kFwdSmemT)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_adj2t<M, false>, at, (int)kAdjSmemT)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_adj2t<M, true>, at, (int)kAdjSmemT);
}

template <int M, bool WIN>
cudaError_t launch_fwd_MW(const Step2D &a, dim3 grid, bool born, bool bands, bool hess, cudaStream_t s)
{
    if (born) return launch_fwd_t<M, true, false, false, WIN>(a, grid, s);
    if (bands && hess) return launch_fwd_t<M, false, true, true, WIN>(a, grid, s);
    if (bands) return launch_fwd_t<M, false, true, false, WIN>(a, grid, s);
    if (hess) return launch_fwd_t<M, false, false, true, WIN>(a, grid, s);
    return launch_fwd_t<M, false, false, false, WIN>(a, grid, s);
}

template <int M>
cudaError_t launch_fwd_M(const Step2D &a, int batch, bool born, bool bands, bool hess, cudaStream_t s,
                         const Maps2D *maps)
{
    dim3 grid((a.g.Nx + Cols<M>::TXO - 1) / Cols<M>::TXO, (a.g.Nz + a.tzc - 1) / a.tzc, batch);
    if (born && maps && !a.win_nx) {
        if (!a.err) return cudaErrorInvalidValue;
        Fwd2T p;
        p.a = a;
        p.m = *maps;
        if (a.g.fs) k_fwd2t<M, true><<<grid, NTH, kFwdSmemT, s>>>(p);
        else k_fwd2t<M, false><<<grid, NTH, kFwdSmemT, s>>>(p);
        return cudaGetLastError();
    }
    if (a.win_nx) return launch_fwd_MW<M, true>(a, grid, born, bands, hess, s);
    return launch_fwd_MW<M, false>(a, grid, born, bands, hess, s);
}

template <int M>
cudaError_t launch_adj_M(const Step2D &a, const Maps2D *maps, int batch, cudaStream_t s)
{
    dim3 grid((a.g.Nx + Cols<M>::TXO - 1) / Cols<M>::TXO, (a.g.Nz + a.tzc - 1) / a.tzc, batch);
    const bool w = a.win_nx != nullptr, f = a.g.fs != 0;
    if (maps && !w) {
        if (!a.err) return cudaErrorInvalidValue;
        Adj2T p;
        p.a = a;
        p.m = *maps;
        if (f) k_adj2t<M, true><<<grid, NTH, kAdjSmemT, s>>>(p);
        else k_adj2t<M, false><<<grid, NTH, kAdjSmemT, s>>>(p);
        return cudaGetLastError();
    }
    if (w && f) k_adj2d<M, true, true><<<grid, NTH, kAdjStageBytes, s>>>(a);
    else if (w) k_adj2d<M, true, false><<<grid, NTH, kAdjStageBytes, s>>>(a);
    else if (f) k_adj2d<M, false, true><<<grid, NTH, kAdjStageBytes, s>>>(a);
    else k_adj2d<M, false, false><<<grid, NTH, kAdjStageBytes, s>>>(a);
    return cudaGetLastError();
}

__global__ void k_window_model(const GridDev gm, const GridDev g, const int *win_x0, const int *win_nx, int shot0,
                               int batch, const float *kdt, const float *binv, const float2 *kd2,
                               const float2 *br2, float *st0, float *st1, long long sstride)
{
    const long long plane = g.plane;
    const long long n = (long long)batch * plane;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int slot = (int)(i / plane);
        const long long c = i - (long long)slot * plane;
        const int z = (int)(c / g.pitch), x = (int)(c - (long long)z * g.pitch);
        const int shot = shot0 + slot;
        const int nxw = win_nx[shot], Nxw = nxw + 2 * g.x0;
        float k = 0.f, b = 0.f;
        float2 k2 = make_float2(0.f, 0.f), b2 = make_float2(0.f, 0.f);
        if (x < Nxw) {
            const int xi = min(max(x - g.x0, 0), nxw - 1);
            const long long cm = (long long)z * gm.pitch + gm.x0 + win_x0[shot] + xi;
            const bool inner = x >= g.x0 && x < g.x0 + nxw;
            k = kdt[cm];
            b = binv[cm];
            if (kd2) {
                k2 = kd2[cm];
                b2 = br2[cm];
                if (!inner) {
                    k2.y = 0.f;
                    b2.y = 0.f;
                }
            }
        }
        for (int q = 0; q < 2; ++q) {
            float *o = (q ? st1 : st0) + slot * sstride;
            o[W_KDT * plane + c] = k;
            o[W_BINV * plane + c] = b;
            if (kd2) {
                reinterpret_cast<float2 *>(o + W_KD2 * plane)[c] = k2;
                reinterpret_cast<float2 *>(o + W_BR2 * plane)[c] = b2;
            }
        }
    }
}

}  // namespace

int march2d_txo(int M) { return M == 2 ? Cols<2>::TXO : Cols<4>::TXO; }

cudaError_t configure_2d_kernels()
{
    cudaError_t e = attr_M<2>();
    if (e != cudaSuccess) return e;
    return attr_M<4>();
}

// Kernel attributes are per device: a flag per device index, set under a
// mutex the first time a thread with that device current asks.
cudaError_t ensure_kernels_configured()
{
    constexpr int kMaxDev = 64;
    static bool done[kMaxDev] = {};
    static std::mutex mu;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    if ((e = configure_2d_kernels()) != cudaSuccess) return e;
    if ((e = configure_3d_kernels()) != cudaSuccess) return e;
    done[dev] = true;
    return cudaSuccess;
}

cudaError_t launch_fwd2d(const Step2D &a, int batch, bool born, bool save_bands, bool hess, cudaStream_t s,
                         const Maps2D *maps)
{
    if (a.g.M == 2) return launch_fwd_M<2>(a, batch, born, save_bands, hess, s, maps);
    return launch_fwd_M<4>(a, batch, born, save_bands, hess, s, maps);
}

cudaError_t launch_adj2d(const Step2D &a, const Maps2D *maps, int batch, cudaStream_t s)
{
    if (a.g.M == 2) return launch_adj_M<2>(a, maps, batch, s);
    return launch_adj_M<4>(a, maps, batch, s);
}

cudaError_t maps2d(Maps2D *m, const GridDev &g, const float *st, long long sstride, const float *kdt,
                   const float *binv, const float2 *kd2, const float2 *br2, const float2 *img, int batch)
{
    // the two model arrays of each kind are one map: their planes must be adjacent
    if (binv != kdt + g.plane || br2 != kd2 + g.plane || sstride % (2 * g.plane)) return cudaErrorInvalidValue;
    m->pps = (int)(sstride / (2 * g.plane));
    m->fps = (int)(sstride / g.plane);
    const cuuint32_t box[3] = {(cuuint32_t)NTH, 1, 1};
    const cuuint64_t s8[2] = {(cuuint64_t)g.pitch * 8, (cuuint64_t)g.plane * 8};
    const cuuint64_t s4[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.plane * 4};
    const cuuint64_t dpr[3] = {(cuuint64_t)g.Nx, (cuuint64_t)g.Nz, (cuuint64_t)batch * m->pps};
    const cuuint64_t dfl[3] = {(cuuint64_t)g.Nx, (cuuint64_t)g.Nz, (cuuint64_t)batch * m->fps};
    const cuuint64_t dmd[3] = {(cuuint64_t)g.Nx, (cuuint64_t)g.Nz, 2};
    const cuuint64_t dim[3] = {(cuuint64_t)g.Nx, (cuuint64_t)g.Nz, (cuuint64_t)batch};
    cudaError_t e;
    if ((e = encode_tmap(&m->pr, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, st, dpr, s8, box)) != cudaSuccess) return e;
    if ((e = encode_tmap(&m->fl, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, st, dfl, s4, box)) != cudaSuccess) return e;
    if ((e = encode_tmap(&m->md, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, kdt, dmd, s4, box)) != cudaSuccess) return e;
    if ((e = encode_tmap(&m->mb, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, kd2, dmd, s8, box)) != cudaSuccess) return e;
    return encode_tmap(&m->im, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, img, dim, s8, box);
}

cudaError_t launch_window_model(const GridDev &gm, const GridDev &g, const int *win_x0, const int *win_nx,
                                int shot0, int batch, const float *kdt, const float *binv, const float2 *kd2,
                                const float2 *br2, float *st0, float *st1, long long sstride, cudaStream_t s)
{
    long long n = batch * g.plane;
    int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 16);
    k_window_model<<<blocks, 256, 0, s>>>(gm, g, win_x0, win_nx, shot0, batch, kdt, binv, kd2, br2, st0, st1,
                                          sstride);
    return cudaGetLastError();
}

cudaError_t launch_pack_adjoint(const GridDev &g, const float *final_state, int shot0, int batch, float *st,
                                long long sstride, cudaStream_t s)
{
    long long n = batch * g.plane;
    int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 16);
    k_pack_adj<<<blocks, 256, 0, s>>>(g, final_state, shot0, batch, st, sstride);
    return cudaGetLastError();
}

}  // namespace lsrtm
