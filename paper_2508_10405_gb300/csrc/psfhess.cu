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
// k_psfh_apply<MASK, TR>: one thread per output pixel, CTAs of 32 x 8 pixels.
//   The input planes over the tile plus a half-wide halo and the corner
//   tables of the halo's rows and columns sit in shared memory; the node
//   windows are read through L1 (a warp's 32 pixels touch at most a few nodes).
//   TR = false: y(r) = sum_a H(r, r - a) x(r - a), the columns gathered at r;
//   TR = true:  y(c) = sum_a H(c + a, c) x(c + a), the transpose.
#include <cuda_runtime.h>

#include <algorithm>

#include "lsrtm_internal.cuh"

namespace lsrtm {

namespace {

constexpr int kTX = 32, kTZ = 8, kThreads = kTX * kTZ;

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

__device__ __forceinline__ float4 fma4(float w, float4 e, float4 acc)
{
    return make_float4(fmaf(w, e.x, acc.x), fmaf(w, e.y, acc.y), fmaf(w, e.z, acc.z), fmaf(w, e.w, acc.w));
}

// Block (i, j) of a packed float4: component 2 i + j.
template <int B>
__device__ __forceinline__ float comp(float4 e)
{
    return B == 0 ? e.x : B == 1 ? e.y : B == 2 ? e.z : e.w;
}

template <int MASK, bool TR>
__global__ void __launch_bounds__(kThreads) k_psfh_apply(const PsfHessDev a, const float *__restrict__ in,
                                                          float *__restrict__ out)
{
    constexpr int NP = MASK == 3 ? 2 : 1;
    constexpr int P0 = MASK == 2 ? 1 : 0;    // first plane in the mask
    constexpr int BM = MASK == 2 ? 3 : 0;    // the block of a single-parameter mask
    extern __shared__ __align__(16) float sm[];
    const int h = a.half, L = 2 * h + 1, LL = L * L;
    const int TRW = kTZ + 2 * h, TCW = kTX + 2 * h;
    float *tile = sm;                                                  // [NP][TRW][TCW]
    Corner *zc = reinterpret_cast<Corner *>(tile + NP * TRW * TCW);    // [TRW]
    Corner *xc = zc + TRW;                                             // [TCW]
    const int t = threadIdx.x, tx = t % kTX, tz = t / kTX;
    const int R0 = (int)blockIdx.y * kTZ, X0 = (int)blockIdx.x * kTX;
    const long long plane = (long long)a.nz * a.nx;

    for (int i = t; i < NP * TRW * TCW; i += kThreads) {
        const int q = i / (TRW * TCW), rem = i - q * TRW * TCW, r = rem / TCW, c = rem - r * TCW;
        const int gz = R0 - h + r, gx = X0 - h + c;
        tile[i] = (gz >= 0 && gz < a.nz && gx >= 0 && gx < a.nx)
                      ? in[(P0 + q) * plane + (long long)gz * a.nx + gx]
                      : 0.f;
    }
    for (int i = t; i < TRW + TCW; i += kThreads) {
        if (i < TRW) zc[i] = corner_of(R0 - h + i, a.nz, a.s, a.nkz);
        else xc[i - TRW] = corner_of(X0 - h + (i - TRW), a.nx, a.s, a.nkx);
    }
    __syncthreads();
    const int rz = R0 + tz, rx = X0 + tx;
    if (rz >= a.nz || rx >= a.nx) return;

    const float4 *pt = a.pt;
    const float *pt1 = reinterpret_cast<const float *>(a.pt);
    const int nkx = a.nkx;
    float acc0 = 0.f, acc1 = 0.f;
    const float *t0 = tile, *t1 = tile + (NP - 1) * TRW * TCW;

    if (!TR) {
        // y(r) = sum_a [sum_corners(c) w P(a)] x(c), c = r - a
        for (int dz = -h; dz <= h; ++dz) {
            const int cz = rz - dz;
            if (cz < 0 || cz >= a.nz) continue;
            const int row = tz + h - dz;
            const Corner Z = zc[row];
            const int z0 = Z.k0 * nkx, z1 = Z.k1 * nkx;
            const float wz1 = Z.w, wz0 = 1.f - Z.w;
            const int arow = (dz + h) * L + h;
            for (int dx = -h; dx <= h; ++dx) {
                const int col = tx + h - dx;
                const int xk0 = xc[col].k0, xk1 = xc[col].k1;
                const float wx1 = xc[col].w, wx0 = 1.f - wx1;
                const int ai = arow + dx;
                const int i00 = (z0 + xk0) * LL + ai, i01 = (z0 + xk1) * LL + ai;
                const int i10 = (z1 + xk0) * LL + ai, i11 = (z1 + xk1) * LL + ai;
                const float w00 = wz0 * wx0, w01 = wz0 * wx1, w10 = wz1 * wx0, w11 = wz1 * wx1;
                const float x0 = t0[row * TCW + col];
                if (MASK == 3) {
                    const float x1 = t1[row * TCW + col];
                    float4 C = make_float4(0.f, 0.f, 0.f, 0.f);
                    C = fma4(w00, __ldg(pt + i00), C);
                    C = fma4(w01, __ldg(pt + i01), C);
                    C = fma4(w10, __ldg(pt + i10), C);
                    C = fma4(w11, __ldg(pt + i11), C);
                    acc0 = fmaf(comp<0>(C), x0, fmaf(comp<1>(C), x1, acc0));
                    acc1 = fmaf(comp<2>(C), x0, fmaf(comp<3>(C), x1, acc1));
                } else {
                    float C = w00 * __ldg(pt1 + 4 * i00 + BM);
                    C = fmaf(w01, __ldg(pt1 + 4 * i01 + BM), C);
                    C = fmaf(w10, __ldg(pt1 + 4 * i10 + BM), C);
                    C = fmaf(w11, __ldg(pt1 + 4 * i11 + BM), C);
                    acc0 = fmaf(C, x0, acc0);
                }
            }
        }
    } else {
        // y(c) = sum_a [sum_corners(c) w P(a)] x(c + a)
        const Corner Z = zc[tz + h], X = xc[tx + h];
        const float w00 = (1.f - Z.w) * (1.f - X.w), w01 = (1.f - Z.w) * X.w;
        const float w10 = Z.w * (1.f - X.w), w11 = Z.w * X.w;
        const int b00 = (Z.k0 * nkx + X.k0) * LL, b01 = (Z.k0 * nkx + X.k1) * LL;
        const int b10 = (Z.k1 * nkx + X.k0) * LL, b11 = (Z.k1 * nkx + X.k1) * LL;
        for (int dz = -h; dz <= h; ++dz) {
            const int row = tz + h + dz;
            const int arow = (dz + h) * L + h;
            for (int dx = -h; dx <= h; ++dx) {
                const int col = tx + h + dx;
                const int ai = arow + dx;
                const float y0 = t0[row * TCW + col];
                if (MASK == 3) {
                    const float y1 = t1[row * TCW + col];
                    float4 C = make_float4(0.f, 0.f, 0.f, 0.f);
                    C = fma4(w00, __ldg(pt + b00 + ai), C);
                    C = fma4(w01, __ldg(pt + b01 + ai), C);
                    C = fma4(w10, __ldg(pt + b10 + ai), C);
                    C = fma4(w11, __ldg(pt + b11 + ai), C);
                    acc0 = fmaf(comp<0>(C), y0, fmaf(comp<2>(C), y1, acc0));
                    acc1 = fmaf(comp<1>(C), y0, fmaf(comp<3>(C), y1, acc1));
                } else {
                    float C = w00 * __ldg(pt1 + 4 * (b00 + ai) + BM);
                    C = fmaf(w01, __ldg(pt1 + 4 * (b01 + ai) + BM), C);
                    C = fmaf(w10, __ldg(pt1 + 4 * (b10 + ai) + BM), C);
                    C = fmaf(w11, __ldg(pt1 + 4 * (b11 + ai) + BM), C);
                    acc0 = fmaf(C, y0, acc0);
                }
            }
        }
    }
    const long long o = (long long)rz * a.nx + rx;
    if (MASK == 3) {
        out[o] = acc0;
        out[plane + o] = acc1;
    } else {
        out[P0 * plane + o] = acc0;
        out[(1 - P0) * plane + o] = 0.f;
    }
}

size_t apply_smem(int mask, int half)
{
    const int np = mask == 3 ? 2 : 1;
    const size_t rows = kTZ + 2 * half, cols = kTX + 2 * half;
    return np * rows * cols * sizeof(float) + (rows + cols) * sizeof(Corner);
}

template <int MASK, bool TR>
cudaError_t launch_t(const PsfHessDev &a, const float *in, float *out, cudaStream_t s)
{
    const size_t sm = apply_smem(MASK, a.half);
    dim3 grid((a.nx + kTX - 1) / kTX, (a.nz + kTZ - 1) / kTZ);
    k_psfh_apply<MASK, TR><<<grid, kThreads, sm, s>>>(a, in, out);
    return cudaGetLastError();
}

}  // namespace

int psfh_max_half() { return kPsfHessMaxHalf; }

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
    case 2: return launch_t<1, false>(a, in, out, s);
    case 3: return launch_t<1, true>(a, in, out, s);
    case 4: return launch_t<2, false>(a, in, out, s);
    case 5: return launch_t<2, true>(a, in, out, s);
    case 6: return launch_t<3, false>(a, in, out, s);
    case 7: return launch_t<3, true>(a, in, out, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lsrtm
