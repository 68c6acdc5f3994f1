// Interpolated PSF Hessian (App. D) on the GPU.
//
// The PSF image L^T L comb of a spike comb (nodes s/2 + k s along both axes)
// holds a localised column of the Hessian around every node. The column at a
// point c between the nodes is the bilinear interpolation (Eq. trilinear in
// its 2D form) of the windows of the four surrounding nodes, each taken
// relative to its own node:
//     H(c + a, c) = sum_corners w_corner(c) P_corner(a),  |a_z|, |a_x| <= half,
//     P_k(a) = Q(node_k + a) (0 outside the image),
// with the 1D weights (1 - w, w), w = (c - node_k0) / s, between the first and
// the last node and a single node (w = 0) beyond them. Two parameters give
// 2 x 2 blocks: block (i, j) takes plane i of the PSF of the comb in
// parameter j. The parameter mask restricts the operator to P H P.
//
// k_psfh_patches: the node windows, packed per (node, offset) as one float4
//   of the four blocks (00, 01, 10, 11), so one 16-byte load serves all four.
// k_psfh_apply<MASK, TR, R>: one thread per output column and R consecutive
//   rows (R = the largest of 8, 4, 2, 1 not above s), CTAs of 32 columns x
//   2 R rows (small CTAs spread the one wave evenly over the SMs). The input
//   planes over the tile plus a half-wide halo and the corner tables of the
//   halo's rows and columns sit in shared memory. Per
//   window offset a thread reads the six node windows covering its rows
//   (three node rows, two node columns; R <= s rows cross at most one node
//   row) through L1, interpolates along x once and along z per row: one
//   loaded value serves R pixels, which keeps the L1 return path (the limit
//   of a one-pixel-per-thread form) below the FMA pipe.
//   TR = false: y(r) = sum_a H(r, r - a) x(r - a), the columns gathered at r;
//   TR = true:  y(c) = sum_a H(c + a, c) x(c + a), the transpose.
// k_psfh3_patches, k_psfh3_rows: the same for 3D images, with the eight
//   corners of Eq. (trilinear) and (y, x) columns of R z rows.
#include <cuda_runtime.h>

#include <algorithm>

#include "lsrtm_internal.cuh"
#include "psfhess3d.cuh"

namespace lsrtm {

namespace {

constexpr int kTX = 32;

struct Corner {
    int k0, k1;
    float w;
};

// Corner nodes and weight of coordinate c (clamped into [0, n)) on an axis
// with nk nodes at s/2 + k s.
__device__ __forceinline__ Corner corner_of(int c, int n, int s, int nk)
{
    c = min(max(c, 0), n - 1);
    const int c0 = s >> 1, last = c0 + (nk - 1) * s;
    Corner r;
    if (c <= c0) {
        r.k0 = r.k1 = 0;
        r.w = 0.f;
    } else if (c >= last) {
        r.k0 = r.k1 = nk - 1;
        r.w = 0.f;
    } else {
        const int k = (c - c0) / s;
        r.k0 = k;
        r.k1 = k + 1;
        r.w = (float)(c - c0 - k * s) / (float)s;
    }
    return r;
}

__global__ void k_psfh_patches(const float *psf_vp, const float *psf_ip, int nz, int nx, int s, int half,
                               int nkz, int nkx, int mask, float4 *pt)
{
    const int L = 2 * half + 1, LL = L * L;
    const long long plane = (long long)nz * nx;
    const long long n = (long long)nkz * nkx * LL;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int node = (int)(i / LL), ai = (int)(i - (long long)node * LL);
        const int kz = node / nkx, kx = node - kz * nkx;
        const int z = (s >> 1) + kz * s + ai / L - half;
        const int x = (s >> 1) + kx * s + ai % L - half;
        const bool inside = z >= 0 && z < nz && x >= 0 && x < nx;
        float v[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int po = b >> 1, pi = b & 1;   // output plane, input (comb) plane
            const float *src = pi ? psf_ip : psf_vp;
            const bool use = inside && src && ((mask >> po) & 1) && ((mask >> pi) & 1);
            v[b] = use ? src[po * plane + (long long)z * nx + x] : 0.f;
        }
        pt[i] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// Parameter-block values: a float4 of the four blocks (two parameters) or
// the one block of a single-parameter mask.
template <int MASK>
struct Blk {
    using T = float;
};
template <>
struct Blk<3> {
    using T = float4;
};

template <int BM>
__device__ __forceinline__ float load_blk(const float4 *pt, int i, float)
{
    return __ldg(reinterpret_cast<const float *>(pt) + 4 * i + BM);
}
template <int BM>
__device__ __forceinline__ float4 load_blk(const float4 *pt, int i, float4)
{
    return __ldg(pt + i);
}
// p0 + w (p1 - p0)
__device__ __forceinline__ float lerp_(float p0, float p1, float w) { return fmaf(w, p1 - p0, p0); }
__device__ __forceinline__ float4 lerp_(float4 p0, float4 p1, float w)
{
    return make_float4(lerp_(p0.x, p1.x, w), lerp_(p0.y, p1.y, w), lerp_(p0.z, p1.z, w), lerp_(p0.w, p1.w, w));
}
__device__ __forceinline__ float sub_(float a, float b) { return a - b; }
__device__ __forceinline__ float4 sub_(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
// q0 + b d1 + c d2 (= (1 - b - c) q0 + b q1 + c q2 with d1 = q1 - q0, d2 = q2 - q0)
__device__ __forceinline__ float mix3(float q0, float d1, float d2, float b, float c)
{
    return fmaf(c, d2, fmaf(b, d1, q0));
}
__device__ __forceinline__ float4 mix3(float4 q0, float4 d1, float4 d2, float b, float c)
{
    return make_float4(mix3(q0.x, d1.x, d2.x, b, c), mix3(q0.y, d1.y, d2.y, b, c), mix3(q0.z, d1.z, d2.z, b, c),
                       mix3(q0.w, d1.w, d2.w, b, c));
}

// Weights of R consecutive rows (first corner row kf) on the node rows
// kf + 1 and kf + 2 (the rest, on kf, is implied): row r puts 1 - w on its k0
// and w on its k1. R <= s keeps every k0 in {kf, kf + 1} and every k1 in
// {kf, .., kf + 2}.
template <int R>
__device__ __forceinline__ void row_weights(const Corner *zc, int kf, float (&wb)[R], float (&wc)[R])
{
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const Corner Z = zc[r];
        const int s0 = Z.k0 - kf, s1 = Z.k1 - kf;
        const float u = 1.f - Z.w, w = Z.w;
        wb[r] = (s0 == 1 ? u : 0.f) + (s1 == 1 ? w : 0.f);
        wc[r] = s1 == 2 ? w : 0.f;
    }
}

// One thread per column and R consecutive rows; CTAs of 32 columns x kRowThreads
// thread rows (32 x kRowThreads R pixels). Per window offset a thread loads the
// six node windows (three node rows x two node columns) that cover its R
// rows, interpolates along x once, then along z per row, so a loaded value
// serves R pixels.
constexpr int kRowThreads = 2, kApplyThreads = kTX * kRowThreads;

template <int MASK, bool TR, int R>
__global__ void __launch_bounds__(kApplyThreads) k_psfh_apply(const PsfHessDev a, const float *__restrict__ in,
                                                               float *__restrict__ out)
{
    using V = typename Blk<MASK>::T;
    constexpr int NP = MASK == 3 ? 2 : 1;
    constexpr int P0 = MASK == 2 ? 1 : 0;    // first plane in the mask
    constexpr int BM = MASK == 2 ? 3 : 0;    // the block of a single-parameter mask
    constexpr int TZ = kRowThreads * R;      // rows of the CTA tile
    extern __shared__ __align__(16) float sm[];
    const int h = a.half, L = 2 * h + 1, LL = L * L;
    const int TRW = TZ + 2 * h, TCW = kTX + 2 * h;
    float *tile = sm;   // [TRW][TCW] of the input, plane pairs interleaved for two parameters
    Corner *zc = reinterpret_cast<Corner *>(tile + NP * TRW * TCW);    // [TRW]
    Corner *xc = zc + TRW;                                             // [TCW]
    const int t = threadIdx.x, tx = t % kTX, ty = t / kTX;
    const int Z0 = (int)blockIdx.y * TZ, X0 = (int)blockIdx.x * kTX;
    const long long plane = (long long)a.nz * a.nx;

    for (int i = t; i < TRW * TCW; i += kApplyThreads) {
        const int r = i / TCW, c = i - r * TCW;
        const int gz = Z0 - h + r, gx = X0 - h + c;
        const bool ok = gz >= 0 && gz < a.nz && gx >= 0 && gx < a.nx;
        const long long g = ok ? (long long)gz * a.nx + gx : 0;
        if (MASK == 3)
            reinterpret_cast<float2 *>(tile)[i] = ok ? make_float2(in[g], in[plane + g]) : make_float2(0.f, 0.f);
        else
            tile[i] = ok ? in[P0 * plane + g] : 0.f;
    }
    for (int i = t; i < TRW + TCW; i += kApplyThreads) {
        if (i < TRW) zc[i] = corner_of(Z0 - h + i, a.nz, a.s, a.nkz);
        else xc[i - TRW] = corner_of(X0 - h + (i - TRW), a.nx, a.s, a.nkx);
    }
    __syncthreads();
    const int rz0 = Z0 + ty * R, rx = X0 + tx;   // this thread: rows rz0 .. rz0 + R - 1, column rx
    if (rz0 >= a.nz || rx >= a.nx) return;

    const float4 *pt = a.pt;
    const int nkx = a.nkx, nkz1 = a.nkz - 1;
    const float2 *t2 = reinterpret_cast<const float2 *>(tile);
    const V zero = V{};
    float acc0[R], acc1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc0[r] = acc1[r] = 0.f;
    float wb[R], wc[R];

    if (!TR) {
        // y(r) = sum_a [sum_corners(c) w P(a)] x(c), c = r - a: for offset
        // row dz the thread's input rows c are rz0 - dz .. + R - 1
        for (int dz = -h; dz <= h; ++dz) {
            const int row0 = ty * R + h - dz;   // tile row of c = rz0 - dz
            const int kf = zc[row0].k0;
            row_weights<R>(zc + row0, kf, wb, wc);
            const int n0 = kf * nkx, n1 = min(kf + 1, nkz1) * nkx, n2 = min(kf + 2, nkz1) * nkx;
            const int arow = (dz + h) * L + h;
            // node values of offset dx = -h, then of dx + 1 while dx is used
            int col = tx + 2 * h;
            int xk0 = xc[col].k0, xk1 = xc[col].k1;
            float wx = xc[col].w;
            V p00 = load_blk<BM>(pt, (n0 + xk0) * LL + arow - h, zero);
            V p01 = load_blk<BM>(pt, (n0 + xk1) * LL + arow - h, zero);
            V p10 = load_blk<BM>(pt, (n1 + xk0) * LL + arow - h, zero);
            V p11 = load_blk<BM>(pt, (n1 + xk1) * LL + arow - h, zero);
            V p20 = load_blk<BM>(pt, (n2 + xk0) * LL + arow - h, zero);
            V p21 = load_blk<BM>(pt, (n2 + xk1) * LL + arow - h, zero);
            for (int dx = -h; dx <= h; ++dx) {
                const int dn = min(dx + 1, h), cn = tx + h - dn, an = arow + dn;
                const int yk0 = xc[cn].k0, yk1 = xc[cn].k1;
                const float wn = xc[cn].w;
                const V n00 = load_blk<BM>(pt, (n0 + yk0) * LL + an, zero);
                const V n01 = load_blk<BM>(pt, (n0 + yk1) * LL + an, zero);
                const V n10 = load_blk<BM>(pt, (n1 + yk0) * LL + an, zero);
                const V n11 = load_blk<BM>(pt, (n1 + yk1) * LL + an, zero);
                const V n20 = load_blk<BM>(pt, (n2 + yk0) * LL + an, zero);
                const V n21 = load_blk<BM>(pt, (n2 + yk1) * LL + an, zero);
                const V q0 = lerp_(p00, p01, wx), q1 = lerp_(p10, p11, wx), q2 = lerp_(p20, p21, wx);
                const V d1 = sub_(q1, q0), d2 = sub_(q2, q0);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const V C = mix3(q0, d1, d2, wb[r], wc[r]);
                    const int o = (row0 + r) * TCW + col;
                    if constexpr (MASK == 3) {
                        const float2 xv = t2[o];
                        acc0[r] = fmaf(C.x, xv.x, fmaf(C.y, xv.y, acc0[r]));
                        acc1[r] = fmaf(C.z, xv.x, fmaf(C.w, xv.y, acc1[r]));
                    } else {
                        acc0[r] = fmaf(C, tile[o], acc0[r]);
                    }
                }
                p00 = n00, p01 = n01, p10 = n10, p11 = n11, p20 = n20, p21 = n21;
                col = cn, wx = wn;
            }
        }
    } else {
        // y(c) = sum_a [sum_corners(c) w P(a)] x(c + a): the thread's rows c
        // and column are fixed, so are their corners
        const int row0 = ty * R + h;   // tile row of c = rz0
        const int kf = zc[row0].k0;
        row_weights<R>(zc + row0, kf, wb, wc);
        const int xk0 = xc[tx + h].k0, xk1 = xc[tx + h].k1;
        const float wx = xc[tx + h].w;
        const int n0 = kf * nkx, n1 = min(kf + 1, nkz1) * nkx, n2 = min(kf + 2, nkz1) * nkx;
        const int b00 = (n0 + xk0) * LL, b01 = (n0 + xk1) * LL, b10 = (n1 + xk0) * LL;
        const int b11 = (n1 + xk1) * LL, b20 = (n2 + xk0) * LL, b21 = (n2 + xk1) * LL;
        // the window offsets in storage order, the next offset's six node
        // values loaded while the current one is used
        V p00 = load_blk<BM>(pt, b00, zero), p01 = load_blk<BM>(pt, b01, zero);
        V p10 = load_blk<BM>(pt, b10, zero), p11 = load_blk<BM>(pt, b11, zero);
        V p20 = load_blk<BM>(pt, b20, zero), p21 = load_blk<BM>(pt, b21, zero);
        int dz = -h, dx = -h;
        for (int ai = 0; ai < LL; ++ai) {
            const int an = min(ai + 1, LL - 1);
            const V n00 = load_blk<BM>(pt, b00 + an, zero), n01 = load_blk<BM>(pt, b01 + an, zero);
            const V n10 = load_blk<BM>(pt, b10 + an, zero), n11 = load_blk<BM>(pt, b11 + an, zero);
            const V n20 = load_blk<BM>(pt, b20 + an, zero), n21 = load_blk<BM>(pt, b21 + an, zero);
            const V q0 = lerp_(p00, p01, wx), q1 = lerp_(p10, p11, wx), q2 = lerp_(p20, p21, wx);
            const V d1 = sub_(q1, q0), d2 = sub_(q2, q0);
            const int ob = (row0 + dz) * TCW + tx + h + dx;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const V C = mix3(q0, d1, d2, wb[r], wc[r]);
                const int o = ob + r * TCW;
                if constexpr (MASK == 3) {
                    const float2 yv = t2[o];
                    acc0[r] = fmaf(C.x, yv.x, fmaf(C.z, yv.y, acc0[r]));
                    acc1[r] = fmaf(C.y, yv.x, fmaf(C.w, yv.y, acc1[r]));
                } else {
                    acc0[r] = fmaf(C, tile[o], acc0[r]);
                }
            }
            p00 = n00, p01 = n01, p10 = n10, p11 = n11, p20 = n20, p21 = n21;
            if (++dx > h) dx = -h, ++dz;
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int z = rz0 + r;
        if (z >= a.nz) break;
        const long long o = (long long)z * a.nx + rx;
        if (MASK == 3) {
            out[o] = acc0[r];
            out[plane + o] = acc1[r];
        } else {
            out[P0 * plane + o] = acc0[r];
            out[(1 - P0) * plane + o] = 0.f;
        }
    }
}

size_t apply_smem(int mask, int half, int R)
{
    const int np = mask == 3 ? 2 : 1;
    const size_t rows = kRowThreads * R + 2 * half, cols = kTX + 2 * half;
    return np * rows * cols * sizeof(float) + (rows + cols) * sizeof(Corner);
}

template <int MASK, bool TR, int R>
cudaError_t launch_t(const PsfHessDev &a, const float *in, float *out, cudaStream_t s)
{
    const size_t sm = apply_smem(MASK, a.half, R);
    dim3 grid((a.nx + kTX - 1) / kTX, (a.nz + kRowThreads * R - 1) / (kRowThreads * R));
    k_psfh_apply<MASK, TR, R><<<grid, kApplyThreads, sm, s>>>(a, in, out);
    return cudaGetLastError();
}

template <int MASK, bool TR>
cudaError_t launch_r(const PsfHessDev &a, const float *in, float *out, cudaStream_t s)
{
    // rows per thread: the largest of 8, 4, 2, 1 not above the node spacing
    if (a.s >= 8) return launch_t<MASK, TR, 8>(a, in, out, s);
    if (a.s >= 4) return launch_t<MASK, TR, 4>(a, in, out, s);
    if (a.s >= 2) return launch_t<MASK, TR, 2>(a, in, out, s);
    return launch_t<MASK, TR, 1>(a, in, out, s);
}

// ---------------------------------------------------------------------------
// 3D (Eq. trilinear as printed: eight corners, products of the three 1D
// weights). CTAs of 32 x 4 (y, x) columns of R z rows; the corner tables of
// the z, y and x coordinates the CTA's windows reach sit in shared memory,
// inputs and node windows are read through L1.
// ---------------------------------------------------------------------------
constexpr int k3X = 32, k3Y = 4, k3Threads = k3X * k3Y;

__global__ void k_psfh3_patches(const float *psf_vp, const float *psf_ip, const PsfHess3Dev a, float4 *pt)
{
    const int L = 2 * a.half + 1, LL = L * L, LLL = LL * L;
    const long long vol = (long long)a.nz * a.ny * a.nx;
    const long long n = (long long)a.nkz * a.nky * a.nkx * LLL;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int node = (int)(i / LLL), ai = (int)(i - (long long)node * LLL);
        const int kz = node / (a.nky * a.nkx), ky = (node / a.nkx) % a.nky, kx = node % a.nkx;
        const int z = (a.s >> 1) + kz * a.s + ai / LL - a.half;
        const int y = (a.s >> 1) + ky * a.s + (ai / L) % L - a.half;
        const int x = (a.s >> 1) + kx * a.s + ai % L - a.half;
        const bool inside = z >= 0 && z < a.nz && y >= 0 && y < a.ny && x >= 0 && x < a.nx;
        const long long v = inside ? ((long long)z * a.ny + y) * a.nx + x : 0;
        float e[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int po = b >> 1, pi = b & 1;
            const float *src = pi ? psf_ip : psf_vp;
            const bool use = inside && src && ((a.mask >> po) & 1) && ((a.mask >> pi) & 1);
            e[b] = use ? src[po * vol + v] : 0.f;
        }
        pt[i] = make_float4(e[0], e[1], e[2], e[3]);
    }
}

// The 3D kernel with the row blocking of the 2D one: each thread owns one
// (y, x) column and R consecutive z rows (R <= s, so its rows span at most
// three node rows); per window offset it loads the twelve node values
// covering them (3 node rows x 2 x 2), interpolates along x and y once and
// along z per row. Inputs are read through L1.
template <int MASK, bool TR, int R>
__global__ void __launch_bounds__(k3Threads) k_psfh3_rows(const PsfHess3Dev a, const float *__restrict__ in,
                                                           float *__restrict__ out)
{
    using V = typename Blk<MASK>::T;
    constexpr int P0 = MASK == 2 ? 1 : 0;
    constexpr int BM = MASK == 2 ? 3 : 0;
    __shared__ Corner zc[8 + 2 * kPsfHessMaxHalf], yc[k3Y + 2 * kPsfHessMaxHalf], xc[k3X + 2 * kPsfHessMaxHalf];
    const int h = a.half, L = 2 * h + 1, LL = L * L, LLL = LL * L;
    const int t = threadIdx.x, tx = t % k3X, ty = t / k3X;
    const int X0 = (int)blockIdx.x * k3X, Y0 = (int)blockIdx.y * k3Y, Z0 = (int)blockIdx.z * R;
    const int NZ = R + 2 * h, NY = k3Y + 2 * h, NX = k3X + 2 * h;
    for (int i = t; i < NZ + NY + NX; i += k3Threads) {
        if (i < NZ) zc[i] = corner_of(Z0 - h + i, a.nz, a.s, a.nkz);
        else if (i < NZ + NY) yc[i - NZ] = corner_of(Y0 - h + (i - NZ), a.ny, a.s, a.nky);
        else xc[i - NZ - NY] = corner_of(X0 - h + (i - NZ - NY), a.nx, a.s, a.nkx);
    }
    __syncthreads();
    const int y = Y0 + ty, x = X0 + tx;
    if (y >= a.ny || x >= a.nx) return;
    const long long vol = (long long)a.nz * a.ny * a.nx, rowz = (long long)a.ny * a.nx;
    const float *in0 = in + P0 * vol, *in1 = in + vol;
    const float4 *pt = a.pt;
    const int nky = a.nky, nkx = a.nkx, nkz1 = a.nkz - 1;
    const V zero = V{};
    float acc0[R], acc1[R], wb[R], wc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc0[r] = acc1[r] = 0.f;
    if (!TR) {
        for (int dz = -h; dz <= h; ++dz) {
            const int row0 = h - dz;   // zc index of c_z = Z0 - dz
            const int kf = zc[row0].k0;
            row_weights<R>(zc + row0, kf, wb, wc);
            const int nq[3] = {kf, min(kf + 1, nkz1), min(kf + 2, nkz1)};
            for (int dy = -h; dy <= h; ++dy) {
                const int cy = y - dy;
                if (cy < 0 || cy >= a.ny) continue;
                const Corner Y = yc[ty + h - dy];
                for (int dx = -h; dx <= h; ++dx) {
                    const int cx = x - dx;
                    if (cx < 0 || cx >= a.nx) continue;
                    const Corner X = xc[tx + h - dx];
                    const int ai = ((dz + h) * L + (dy + h)) * L + (dx + h);
                    V Q[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const int b0 = (nq[q] * nky + Y.k0) * nkx, b1 = (nq[q] * nky + Y.k1) * nkx;
                        const V v0 = lerp_(load_blk<BM>(pt, (b0 + X.k0) * LLL + ai, zero),
                                           load_blk<BM>(pt, (b0 + X.k1) * LLL + ai, zero), X.w);
                        const V v1 = lerp_(load_blk<BM>(pt, (b1 + X.k0) * LLL + ai, zero),
                                           load_blk<BM>(pt, (b1 + X.k1) * LLL + ai, zero), X.w);
                        Q[q] = lerp_(v0, v1, Y.w);
                    }
                    const V d1 = sub_(Q[1], Q[0]), d2 = sub_(Q[2], Q[0]);
                    const long long cb = (long long)cy * a.nx + cx;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int cz = Z0 + r - dz;
                        if (cz < 0 || cz >= a.nz) continue;
                        const V C = mix3(Q[0], d1, d2, wb[r], wc[r]);
                        const long long c = cz * rowz + cb;
                        if constexpr (MASK == 3) {
                            const float v0 = __ldg(in0 + c), v1 = __ldg(in1 + c);
                            acc0[r] = fmaf(C.x, v0, fmaf(C.y, v1, acc0[r]));
                            acc1[r] = fmaf(C.z, v0, fmaf(C.w, v1, acc1[r]));
                        } else {
                            acc0[r] = fmaf(C, __ldg(in0 + c), acc0[r]);
                        }
                    }
                }
            }
        }
    } else {
        const int kf = zc[h].k0;
        row_weights<R>(zc + h, kf, wb, wc);
        const Corner Y = yc[ty + h], X = xc[tx + h];
        int base[3][2][2];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int kz = min(kf + q, nkz1);
            base[q][0][0] = ((kz * nky + Y.k0) * nkx + X.k0) * LLL;
            base[q][0][1] = ((kz * nky + Y.k0) * nkx + X.k1) * LLL;
            base[q][1][0] = ((kz * nky + Y.k1) * nkx + X.k0) * LLL;
            base[q][1][1] = ((kz * nky + Y.k1) * nkx + X.k1) * LLL;
        }
        for (int dz = -h; dz <= h; ++dz) {
            for (int dy = -h; dy <= h; ++dy) {
                const int cy = y + dy;
                if (cy < 0 || cy >= a.ny) continue;
                for (int dx = -h; dx <= h; ++dx) {
                    const int cx = x + dx;
                    if (cx < 0 || cx >= a.nx) continue;
                    const int ai = ((dz + h) * L + (dy + h)) * L + (dx + h);
                    V Q[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const V v0 = lerp_(load_blk<BM>(pt, base[q][0][0] + ai, zero),
                                           load_blk<BM>(pt, base[q][0][1] + ai, zero), X.w);
                        const V v1 = lerp_(load_blk<BM>(pt, base[q][1][0] + ai, zero),
                                           load_blk<BM>(pt, base[q][1][1] + ai, zero), X.w);
                        Q[q] = lerp_(v0, v1, Y.w);
                    }
                    const V d1 = sub_(Q[1], Q[0]), d2 = sub_(Q[2], Q[0]);
                    const long long cb = (long long)cy * a.nx + cx;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int cz = Z0 + r + dz;
                        if (cz < 0 || cz >= a.nz) continue;
                        const V C = mix3(Q[0], d1, d2, wb[r], wc[r]);
                        const long long c = cz * rowz + cb;
                        if constexpr (MASK == 3) {
                            const float v0 = __ldg(in0 + c), v1 = __ldg(in1 + c);
                            acc0[r] = fmaf(C.x, v0, fmaf(C.z, v1, acc0[r]));
                            acc1[r] = fmaf(C.y, v0, fmaf(C.w, v1, acc1[r]));
                        } else {
                            acc0[r] = fmaf(C, __ldg(in0 + c), acc0[r]);
                        }
                    }
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int z = Z0 + r;
        if (z >= a.nz) break;
        const long long o = z * rowz + (long long)y * a.nx + x;
        if (MASK == 3) {
            out[o] = acc0[r];
            out[vol + o] = acc1[r];
        } else {
            out[P0 * vol + o] = acc0[r];
            out[(1 - P0) * vol + o] = 0.f;
        }
    }
}

template <int MASK, bool TR, int R>
cudaError_t launch3_r(const PsfHess3Dev &a, const float *in, float *out, cudaStream_t s)
{
    dim3 grid((a.nx + k3X - 1) / k3X, (a.ny + k3Y - 1) / k3Y, (a.nz + R - 1) / R);
    k_psfh3_rows<MASK, TR, R><<<grid, k3Threads, 0, s>>>(a, in, out);
    return cudaGetLastError();
}

template <int MASK, bool TR>
cudaError_t launch3_t(const PsfHess3Dev &a, const float *in, float *out, cudaStream_t s)
{
    if (a.s >= 8) return launch3_r<MASK, TR, 8>(a, in, out, s);
    if (a.s >= 4) return launch3_r<MASK, TR, 4>(a, in, out, s);
    if (a.s >= 2) return launch3_r<MASK, TR, 2>(a, in, out, s);
    return launch3_r<MASK, TR, 1>(a, in, out, s);
}

}  // namespace

int psfh_max_half() { return kPsfHessMaxHalf; }

cudaError_t launch_psfh3_patches(const float *psf_vp, const float *psf_ip, const PsfHess3Dev &a, float4 *pt,
                                 cudaStream_t st)
{
    const long long L = 2 * a.half + 1;
    const long long n = (long long)a.nkz * a.nky * a.nkx * L * L * L;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 16);
    k_psfh3_patches<<<blocks, 256, 0, st>>>(psf_vp, psf_ip, a, pt);
    return cudaGetLastError();
}

cudaError_t launch_psfh3_apply(const PsfHess3Dev &a, bool transpose, const float *in, float *out, cudaStream_t s)
{
    switch (a.mask * 2 + (transpose ? 1 : 0)) {
    case 2: return launch3_t<1, false>(a, in, out, s);
    case 3: return launch3_t<1, true>(a, in, out, s);
    case 4: return launch3_t<2, false>(a, in, out, s);
    case 5: return launch3_t<2, true>(a, in, out, s);
    case 6: return launch3_t<3, false>(a, in, out, s);
    case 7: return launch3_t<3, true>(a, in, out, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_psfh_patches(const float *psf_vp, const float *psf_ip, int nz, int nx, int s, int half,
                                int nkz, int nkx, int mask, float4 *pt, cudaStream_t st)
{
    const long long n = (long long)nkz * nkx * (2 * half + 1) * (2 * half + 1);
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    k_psfh_patches<<<blocks, 256, 0, st>>>(psf_vp, psf_ip, nz, nx, s, half, nkz, nkx, mask, pt);
    return cudaGetLastError();
}

cudaError_t launch_psfh_apply(const PsfHessDev &a, bool transpose, const float *in, float *out, cudaStream_t s)
{
    switch (a.mask * 2 + (transpose ? 1 : 0)) {
    case 2: return launch_r<1, false>(a, in, out, s);
    case 3: return launch_r<1, true>(a, in, out, s);
    case 4: return launch_r<2, false>(a, in, out, s);
    case 5: return launch_r<2, true>(a, in, out, s);
    case 6: return launch_r<3, false>(a, in, out, s);
    case 7: return launch_r<3, true>(a, in, out, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lsrtm
