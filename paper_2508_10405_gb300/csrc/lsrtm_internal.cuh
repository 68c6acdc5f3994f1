// Internal declarations shared by the engine and the kernel translation units.
// Layout of every wavefield and model array on the device: padded grid
// Nz x Ny x Nx (interior + npml on each side; Ny = 1 in 2D), x fastest with a
// row pitch that is a multiple of 32 floats, one "plane" = Nz*Ny*pitch floats.
// A shot's state is a block of planes; shots of a batch are consecutive blocks.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lsrtm {

constexpr int kMaxM = 4;

struct GridDev {
    int ndim, M;
    int nz, ny, nx;        // interior
    int Nz, Ny, Nx;        // padded
    int pitch;             // floats per padded row (multiple of 32)
    long long plane;       // floats per field plane
    long long rowz;        // floats between consecutive z (Ny * pitch)
    int z0, y0, x0;        // interior origin in padded coordinates
    float cz[kMaxM], cy[kMaxM], cx[kMaxM];  // c_l / h
    float dt;
    int nt;
    int fs;                // free surface on row z0 (method of images; see lsrtm_config)
    const int *abort;      // non-finite guard word (or null): when nonzero, the
                           // time-step kernels return at once, so the rest of a
                           // tripped time loop costs only its launches
};

// The guard checks the pressure planes of every slot every guard_interval
// time steps of a loop (kGuardInterval when the configuration gives 0).
constexpr int kGuardInterval = 64;
// Guard codes: (loop kind << 24) | (time step or CG iteration + 1).
enum GuardKind { GK_BACKGROUND = 1, GK_BORN = 2, GK_MIGRATION = 3, GK_MODELLING = 4, GK_RECOMPUTE = 5,
                 GK_CG = 6 };
__host__ __device__ inline int guard_code(int kind, int n) { return (kind << 24) | ((n + 1) & 0xFFFFFF); }
#ifdef __CUDACC__
__device__ __forceinline__ bool guard_tripped(const GridDev &g) { return g.abort && *g.abort; }
#endif

// Free surface: the padded row a ghost node row r < z0 mirrors (p odd about
// z0), and the half row a ghost half row k < z0 mirrors (v_z even).
__host__ __device__ inline int fs_node_row(const GridDev &g, int r) { return 2 * g.z0 - r; }
__host__ __device__ inline int fs_half_row(const GridDev &g, int k) { return 2 * g.z0 - 1 - k; }

// CPML coefficients, per direction d (0 z, 1 y, 2 x) and array: a/b at
// integer nodes (ai, bi) and at half nodes (ah, bh).
struct Pml {
    const float *ai[3], *bi[3], *ah[3], *bh[3];
};

// Boundary-band geometry (per shot, per step): the p band and the normal-v
// band each hold NB values laid out as strips:
//   2D: [x-left M*nz][x-right M*nz][z-top M*nx][z-bottom M*nx]
//   3D: [x-faces 2*M*nz*ny][y-faces 2*M*nz*nx][z-faces 2*M*ny*nx]
// The buffers hold steps [t0, t0 + nsteps) of shots [shot0, ...): the band of
// shot s at step n starts at ((s - shot0) * nsteps + (n - t0)) * NB.
//
// Storage: FP32, or 16-bit values with one FP32 scale per band per step
// (BF16 or FP16). With a 16-bit format the time-step kernels write the step's
// bands in FP32 into a per-slot stage; k_band_pack then takes the largest
// magnitude of each band, stores scale = pow2_scale(max) and the values
// divided by it (so FP16 keeps its full mantissa down to about 2^-23 of the
// band's maximum), and the reverse pass multiplies back.
enum BandFmt { BAND_F32 = 0, BAND_BF16S = 1, BAND_F16S = 2 };

struct Bands {
    void *p;              // [shots][nsteps][NB]
    void *v;              // [shots][nsteps][NB]
    long long nb;         // NB
    int fmt;              // BandFmt
    int shot0, t0, nsteps;
    float *scale;         // [shots][nsteps][2] (p, v) scales (16-bit formats)
    float *stage;         // [batch][2][NB] FP32 bands of the current step (16-bit formats)
};

// Band row (shot, step) within the buffers.
__host__ __device__ inline long long band_row(const Bands &b, int shot, int n)
{
    return (long long)(shot - b.shot0) * b.nsteps + (n - b.t0);
}

__host__ __device__ inline long long band_base(const Bands &b, int shot, int n) { return band_row(b, shot, n) * b.nb; }

#ifdef __CUDACC__
// Scale of a 16-bit block (a band of one step, a checkpoint plane) whose
// largest magnitude is m: the power of two 2^e with m / 2^e in [2^14, 2^15),
// so the scaled values fit FP16 and BF16 alike and the division and the
// multiplication back are exact; e >= -126 keeps the scale and its inverse
// normal (a block of subnormal magnitudes is then stored below 2^14). A zero
// block gets 1.
__device__ __forceinline__ float pow2_scale(float m)
{
    if (!(m > 0.f)) return 1.f;
    return ldexpf(1.f, max(ilogbf(m) - 14, -126));
}

// Saves value v at slot idx of field (0: p band, 1: normal-v band) of the band
// starting at base = band_base(shot, n) of batch slot `slot`.
__device__ __forceinline__ void band_put(const Bands &b, int field, int slot, long long base, long long idx, float v)
{
    if (b.fmt == BAND_F32) reinterpret_cast<float *>(field ? b.v : b.p)[base + idx] = v;
    else b.stage[((long long)slot * 2 + field) * b.nb + idx] = v;
}

// Value at slot idx of field of the band in row `row` (band_row(shot, n)).
__device__ __forceinline__ float band_get(const Bands &b, int field, long long row, long long idx)
{
    const long long o = row * b.nb + idx;
    const void *base = field ? b.v : b.p;
    if (b.fmt == BAND_F32) return reinterpret_cast<const float *>(base)[o];
    const float sc = b.scale[row * 2 + field];
    if (b.fmt == BAND_BF16S) return sc * __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(base)[o]);
    return sc * __half2float(reinterpret_cast<const __half *>(base)[o]);
}
#endif

// Receivers grouped by (shot, tile): CSR over shot*ntiles + tile.
struct TileRecs {
    const int *ptr;       // [nshot*ntiles + 1]
    const int2 *rec;      // (cell offset in plane, global receiver row), sorted by cell
    int ntiles;           // tiles per shot
};

// Arguments of the fused 2D time-step kernels.
struct Step2D {
    GridDev g;
    Pml pml;
    const float *kdt;     // dt * kappa          [plane]
    const float *binv;    // 1 / rho             [plane]
    const float2 *kd2;    // (dt kappa, dt kappa dln kappa) [plane] (Born only)
    const float2 *br2;    // (1/rho, dln rho / rho)        [plane] (Born only)
    const float *in;      // ping state, shot slot s at in + s*sstride
    float *out;           // pong state
    float *psiv;          // in-place node CPML memories, slot stride vstride
    long long sstride, vstride;
    int n;                // time step
    int tzc;              // rows of the z-chunk each CTA marches through
    int shot0;            // global index of slot 0
    const float *wav;     // [nt] or [nshot][nt]
    int wav_per_shot;
    const int *src_cell;  // [nshot] plane offset of the source node
    float src_scale;      // dt / cell volume
    TileRecs trec;
    float *dstage;        // [nrec_total][nt]: records (forward) or residual (adjoint)
    int rec_bg;           // forward: record the background p instead of dp (nonlinear modelling)
    Bands bands;
    float *hess;          // [batch][plane] pseudo-Hessian accumulators (or null)
    float2 *img;          // [batch][plane] image accumulators (adjoint)
    // Aperture windows (null: every shot spans the whole model). A windowed
    // shot runs on its own grid of win_nx[shot] + 2 npml columns; its model
    // planes sit in its slot after the state (kWinStatePlanes2D planes per
    // slot) and its x CPML profiles at pml.*[2] + shot * pml_xstride.
    const int *win_nx;
    int pml_xstride;
    int *err;             // error word of the TMA-staged kernels (1 = a wait gave up, 2 = misaligned copy refused)
};

// Planes of a 2D slot when shots have aperture windows: the 10 state planes,
// then dt kappa, 1/rho and the two Born pairs of the shot's window.
constexpr int kWinStatePlanes2D = 16;

// Arguments of the 3D background time-step kernels (state updated in place).
struct Step3D {
    GridDev g;
    Pml pml;
    const float *kdt, *binv;
    float *st;                // slot 0 of the batch; slot stride sstride floats
    long long sstride;
    int n;
    int shot0;
    const float *wav;
    int wav_per_shot;
    const int *src_cell;
    float src_scale;
    Bands bands;
    float *hess;              // [batch][plane]
    float *dstage;            // pressure records [nrec_total][nt] (nonlinear modelling)
    int rec_bg;               // record the pressure p^{n+1}
    const int *rmap;          // [nshot][plane]: first entry of the node's receivers in rcell/rrow, or -1
    const int *rptr;          // [nshot+1] per-shot ranges of rcell/rrow
    const int *rcell;         // receiver cells, sorted by cell within a shot
    const int *rrow;          // global receiver rows
};

// Fused 3D time-step kernels (kernels3d_fused.cu): CTAs of kTile3X x kTile3Y
// (x, y) columns marching a z-chunk of tzc rows, ping-pong state buffers.
constexpr int kTile3X = 32, kTile3Y = 12;
// Pair-plane offsets within a slot. Born ping-pong: (p, dp), (vx, dvx),
// (vy, dvy), (vz, dvz), (psi_p, dpsi_p) x y z; the node CPML memories
// (psi_v, dpsi_v) x y z live in a separate in-place block.
enum { F3_P = 0, F3_VX = 1, F3_VY = 2, F3_VZ = 3, F3_PPX = 4, F3_PPY = 5, F3_PPZ = 6 };
constexpr int kBornPairs3F = 7;

struct Step3F {
    // TMA descriptors (64-byte aligned, first): the input state's pair planes
    // in four box shapes, the model pair planes (plane 0 kd2, plane 1 br2)
    CUtensorMap in_core, in_wide, in_xbox, in_ybox, m_core, m_ybr;
    GridDev g;
    Pml pml;
    const float *in;          // input state, slot s at in + s * in_pairs pair planes
    float *out;               // output state, slot stride out_pairs pair planes
    float *psiv;              // in-place node CPML memories, slot stride psiv_pairs pair planes
    int in_pairs, out_pairs, psiv_pairs;
    const float2 *br2;        // (1/rho, dln rho / rho), for the first rows of a march
    int n, tzc, shot0;
    const float *wav;
    int wav_per_shot;
    const int *src_cell;
    float src_scale;
    TileRecs trec;            // receivers per (shot, z-chunk, y tile, x tile)
    float *dstage;            // records [nrec_total][nt]
    int *err;                 // error word: 1 = a wait gave up, 2 = a misaligned copy was refused
};
// Fused 3D adjoint layout (float planes of a slot): pairs (p, lambda_p) 0-1,
// (vx, lambda_vx) 2-3, (vy, lambda_vy) 4-5, (vz, lambda_vz) 6-7, then the
// lambda CPML memories psi_p x y z (8-10) and psi_v x y z (11-13).
enum { A3F_PL = 0, A3F_VX = 2, A3F_VY = 4, A3F_VZ = 6, A3F_LPPX = 8, A3F_LPPY = 9, A3F_LPPZ = 10,
       A3F_LPVX = 11, A3F_LPVY = 12, A3F_LPVZ = 13 };
constexpr int kAdjPlanes3F = 14;

struct Adj3F {
    // input-state pair planes (core, wide, xbox, ybox), input-state float
    // planes (core, xwide, ywide, xbox, ybox), model float planes (plane 0
    // dt kappa, plane 1 1/rho: core, wide, ybr)
    CUtensorMap p_core, p_wide, p_xbox, p_ybox;
    CUtensorMap f_core, f_xwide, f_ywide, f_xbox, f_ybox;
    CUtensorMap m_core, m_wide, m_ybr;
    GridDev g;
    Pml pml;
    const float *in;          // input state, slot stride in_planes float planes
    float *out;               // output state, slot stride out_planes
    int in_planes, out_planes;
    const float *kdt, *binv;  // for the first rows of a march
    float2 *img;              // [batch][plane] image accumulators (in place)
    int n, tzc, shot0;
    const float *wav;
    int wav_per_shot;
    const int *src_cell;
    float src_scale;
    Bands bands;
    TileRecs trec;
    const float *dstage;      // residual [nrec_total][nt]
    int *err;
};
cudaError_t fused3d_adj_maps(Adj3F &a, const float *kdt, const float *binv, int batch);
cudaError_t launch_adj3f(const Adj3F &a, int batch, cudaStream_t s);
// (p, 0), (vx, 0), (vy, 0), (vz, 0) into the fused layout from final states
// [p][vz][vy][vx] (shot index fs0 + slot).
cudaError_t launch_pack3f(const GridDev &g, const float *final_state, int fs0, int batch, float *st,
                          long long sstride, cudaStream_t s);
cudaError_t make_tmap3(CUtensorMap *m, const void *base, const GridDev &g, int esz, long long nq, int bx, int by);
cudaError_t fused3d_born_maps(Step3F &a, const float2 *kd2, const float2 *br2, int batch);
size_t fused3d_born_smem(int M);
cudaError_t launch_born3f(const Step3F &a, int batch, cudaStream_t s);

// 3D background launchers (kernels3d.cu). stages: 1 = velocity stage, 2 =
// pressure stage, 3 = both.
cudaError_t launch_fwd3d(const Step3D &a, int batch, bool bands, bool hess, int stages, cudaStream_t s);

// 2D kernels: CTAs of kThreads2D threads, one x-column per thread; a CTA owns
// march2d_txo(M) output columns and a z-chunk of Step2D::tzc rows.
constexpr int kThreads2D = 256;
int march2d_txo(int M);

// Launchers (kernels2d.cu). Return the cudaError of the launch.
struct Maps2D;
// maps (Born modelling only): TMA row staging, as for launch_adj2d.
cudaError_t launch_fwd2d(const Step2D &a, int batch, bool born, bool save_bands, bool hess,
                         cudaStream_t s, const Maps2D *maps = nullptr);
// TMA row maps of the 2D Born and migration kernels reading one state buffer
// (boxes one kThreads2D-wide row of one field): pr over the float2 pair planes
// of every slot (8-byte elements; coordinates x, z, slot * pps + pair), fl
// over its float planes (x, z, slot * fps + plane), md over dt kappa and
// 1/rho (x, z, 0 | 1), mb over the Born model pairs (dt kappa, dt kappa
// dlnk), (1/rho, rr) (x, z, 0 | 1), im over the image accumulators (x, z,
// slot). Outside the padded grid the copies read zeros.
struct Maps2D {
    CUtensorMap pr, fl, md, mb, im;
    int pps, fps;
};
cudaError_t maps2d(Maps2D *m, const GridDev &g, const float *st, long long sstride, const float *kdt,
                   const float *binv, const float2 *kd2, const float2 *br2, const float2 *img, int batch);
// maps: TMA row staging (shots without aperture windows), or null for the
// per-thread asynchronous copies.
cudaError_t launch_adj2d(const Step2D &a, const Maps2D *maps, int batch, cudaStream_t s);
// cuTensorMapEncodeTiled (element strides 1, no swizzle, zero fill).
cudaError_t encode_tmap(CUtensorMap *m, CUtensorMapDataType type, int rank, const void *base, const cuuint64_t *dims,
                        const cuuint64_t *strides, const cuuint32_t *box);
cudaError_t configure_2d_kernels();
cudaError_t configure_3d_kernels();
// Sets the launch attributes (dynamic shared memory limits) of every kernel
// on the current device, once per device; thread safe.
cudaError_t ensure_kernels_configured();
// Copies each windowed shot's model into its slot (both ping-pong buffers):
// column x of the shot's grid takes model column npml + x0 + clamp(x - npml,
// 0, nx_w - 1) of the full padded planes (edge replication of the window);
// the Born perturbation (.y of the pairs) is kept on the window interior only
// and zeroed in its pad; columns beyond the shot's grid are zero.
cudaError_t launch_window_model(const GridDev &gm, const GridDev &g, const int *win_x0, const int *win_nx,
                                int shot0, int batch, const float *kdt, const float *binv, const float2 *kd2,
                                const float2 *br2, float *st0, float *st1, long long sstride, cudaStream_t s);
// Adjoint start state (p, 0), (vx, 0), (vz, 0) from the saved background final states.
cudaError_t launch_pack_adjoint(const GridDev &g, const float *final_state, int shot0, int batch,
                                float *st, long long sstride, cudaStream_t s);

// Nonstationary deblurring filters (deblur.cu): per comb node of spacing s a
// flen x flen filter from FP64 normal equations over the node's window of
// the [2][nz][nx] images, then the valence-weighted filtered image.
// filt: [2][nkz][nkx][flen*flen]; flag |= 1 where a factorisation failed.
int deblur_nodes(int n, int s);
constexpr size_t kDeblurSmemLimit = 227 * 1024;   // dynamic shared memory of one CTA
// Warps of the filter solve that form lag sums (as many as fit; 0: the
// filter length does not fit shared memory).
int deblur_solve_warps(int nz, int nx, int s, int flen);
cudaError_t launch_deblur(const float *mref, const float *mrem, int nz, int nx, int s, int flen, double eps,
                          float *filt, float *out, int *flag, cudaStream_t st);

// Interpolated PSF Hessian (psfhess.cu, App. D): node windows of the PSF
// images, packed per (node, offset) as float4 (blocks 00, 01, 10, 11: output
// plane i, input plane j at component 2 i + j), and the on-the-fly
// application of P H P or P H^T P to a [2][nz][nx] image (mask 1, 2 or 3).
constexpr int kPsfHessMaxHalf = 15;
struct PsfHessDev {
    int nz, nx, s, half, nkz, nkx, mask;
    const float4 *pt;   // [nkz][nkx][(2 half + 1)^2]
};
int psfh_max_half();
cudaError_t launch_psfh_patches(const float *psf_vp, const float *psf_ip, int nz, int nx, int s, int half,
                                int nkz, int nkx, int mask, float4 *pt, cudaStream_t st);
cudaError_t launch_psfh_apply(const PsfHessDev &a, bool transpose, const float *in, float *out, cudaStream_t s);

// Utility kernels (kernels_util.cu).
// 16-bit band formats: per slot and field, scale = pow2_scale(max|stage|) and the
// scaled values into the band store at row band_row(shot0 + slot, n).
cudaError_t launch_band_pack(const Bands &b, int batch, int shot0, int n, cudaStream_t s);
cudaError_t launch_model_prep(const GridDev &g, const float *vp, const float *rho, float *kdt,
                              float *binv, cudaStream_t s);
cudaError_t launch_pert_prep(const GridDev &g, const float *dm, const float *kdt,
                             const float *binv, float2 *kd2, float2 *br2, cudaStream_t s);
// Adds the residual of step n to lambda_p (the .y of the (p, lambda_p) pairs).
cudaError_t launch_inject_residual(const GridDev &g, const TileRecs &tr, int batch, int shot0,
                                   const float *dstage, int n, float2 *pl, long long sstride2,
                                   cudaStream_t s);
// Stacks the batch's per-slot images (grid g) into the FP64 interior image of
// the model grid gm; with aperture windows (win_x0 non-null) slot b covers the
// columns [win_x0, win_x0 + win_nx) of shot shot0 + b.
cudaError_t launch_image_accumulate(const GridDev &gm, const GridDev &g, const float2 *img, int batch, int shot0,
                                    const int *win_x0, const int *win_nx, double2 *acc, cudaStream_t s);
cudaError_t launch_image_finalize(const GridDev &g, const double2 *acc, const float *kdt,
                                  const float *binv, float *gout, cudaStream_t s);
cudaError_t launch_hess_accumulate(const GridDev &gm, const GridDev &g, const float *hess, int batch, int shot0,
                                   const int *win_x0, const int *win_nx, double *acc, cudaStream_t s);
cudaError_t launch_hess_finalize(const GridDev &g, const double *acc, float *out,
                                 cudaStream_t s);
cudaError_t launch_max_abs_reduce(const float *x, long long n, float *out, cudaStream_t s);
cudaError_t launch_nonfinite_count(const float *x, long long n, int *flag, cudaStream_t s);
// Non-finite guard: sets *word to `code` (unless already set) if one of the
// first `count` floats of any of `nslots` slots (slot stride `stride` floats;
// base, count and stride multiples of 4 floats) is NaN or Inf.
cudaError_t launch_guard_state(const float *base, long long stride, long long count, int nslots, int *word,
                               int code, cudaStream_t s);
// 16-bit checkpoint planes (fmt BAND_BF16S or BAND_F16S): planes [p0, p0 +
// planes) of bs slots (slot stride sstride floats, plane floats each) to and
// from a snapshot stored [slot][ck_planes][plane] in 16 bits with one scale
// per slot and plane derived from amax ([slot][ck_planes], the planes'
// largest magnitudes, written by the pack).
cudaError_t launch_ck_pack(const float *src, long long sstride, long long plane, int planes, int p0, int bs,
                           int ck_planes, int fmt, void *dst, float *amax, cudaStream_t s);
cudaError_t launch_ck_unpack(float *dst, long long sstride, long long plane, int planes, int p0, int bs,
                             int ck_planes, int fmt, const void *src, const float *amax, cudaStream_t s);
// The same for n FP64 scalars.
cudaError_t launch_guard_scalars(const double *v, int n, int *word, int code, cudaStream_t s);
// Muted data residual: out = mute(r, n) fo[r] (dobs - dsyn), dsyn nullable; the
// mute is 0 for n < n0[r], then (1 - cos(pi v)) / 2 with v = (n - n0[r]) b + a0[r]
// (1 for v >= 1 or b = 0).
cudaError_t launch_mute_residual(const float *dobs, const float *dsyn, const int *n0, const float *a0,
                                 const float *fo, long long nrec, int nt, float b, float *out, cudaStream_t s);
cudaError_t launch_comb(const GridDev &g, int param, int spacing, float *m, cudaStream_t s);
// rmap[rcell[q]] = q for the first receiver q of each node in [q0, q1) (3D receiver maps).
cudaError_t launch_rmap_scatter(int *rmap, const int *rcell, int q0, int q1, cudaStream_t s);

// FP64-accumulated vector kernels for the Krylov driver.
cudaError_t launch_dot(const float *x, const float *y, long long n, double *out, double *work,
                       cudaStream_t s);
cudaError_t launch_dot_w(const float *x, const float *y, const float *w, long long n,
                         double *out, double *work, cudaStream_t s);
// x += alpha*p, with alpha = num/den read from device scalars (sign: +1 or -1)
cudaError_t launch_axpy_ratio(float *x, const float *p, const double *num, const double *den,
                              float sign, long long n, cudaStream_t s);
// p = z + (num/den) * p
cudaError_t launch_xpby_ratio(float *p, const float *z, const double *num, const double *den,
                              long long n, cudaStream_t s);
cudaError_t launch_mul_mask(float *x, const float *w, int param_mask, long long nint,
                            cudaStream_t s);
cudaError_t launch_scale_copy(float *dst, const float *src, long long n, cudaStream_t s);
cudaError_t launch_precond_build(const float *h, const float *hmax, float eps, long long nint,
                                 float *minv, cudaStream_t s);

}  // namespace lsrtm
