// Nonstationary deblurring filters (App. E) on the GPU.
//
// App. E relates the reference image m' and the remigrated image m'' = H m'
// by a convolution with the inverse of a locally translation-invariant
// Hessian, f * m'' ~= m'. Per comb node k (spacing s, nodes at s/2 + i s) a
// flen x flen FIR filter solves, over the window of pixels within s of the
// node (clipped to the image),
//     min_f  sum_p ((f * m'')(p) - m'(p))^2 + eps_k ||f||^2,
//     (f * g)(p) = sum_{|a|,|b|<=h} f[a,b] g(p - (a,b)), g = 0 outside,
//     eps_k = eps * trace(A^T A) / flen^2,
// through its FP64 normal equations (A^T A + eps_k I) f = A^T m'. The image
// delta m = sum_k w_k (f_k * m_rtm) / sum_k w_k blends the filtered blocks with
// bilinear valence weights w_k(p) = max(0, 1 - |z - z_k|/s) max(0, 1 - |x - x_k|/s).
//
// k_deblur_solve: one CTA per (node, parameter plane). The window's patch of
// m'' (window + h on each side, zero outside the image) sits in shared memory
// as float. Entry (u, v) of A^T A is the sum of P(q) P(q + d) over the window
// shifted to tap u's origin, d = origin(v) - origin(u): the products depend on
// the lag d only, so per lag one warp forms, for every patch row, the
// running sums of the row's lagged products over the window width at every
// origin column (one pass along the row), then slides those along z over the
// window height at every origin row. That is 15x fewer FP64 operations than
// summing each entry over the window (products of two floats are exact in
// FP64; sums in FP64). The matrix, factorised in place by a right-looking
// Cholesky, and the right-hand side stay in shared memory (121 x 121 doubles
// = 117 KB for flen = 11).
// k_deblur_apply: one thread per pixel and plane; FP32 taps, at most four
// covering nodes.
// The paper's own Fourier form of the filter (per-block Wiener ratio) follows
// below the space-domain kernels.
#include <cuda_runtime.h>

#include <algorithm>

#include "lsrtm_internal.cuh"
#include "wiener.cuh"

namespace lsrtm {

namespace {

constexpr int kSolveThreads = 256;

__global__ void __launch_bounds__(kSolveThreads) k_deblur_solve(const float *mref, const float *mrem, int nz,
                                                                 int nx, int s, int flen, double eps,
                                                                 float *filt, int *flag, int nrs)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = flen * flen, h = flen / 2;
    const int nkz = gridDim.y, nkx = gridDim.x;
    const int param = blockIdx.z;
    const int zk = s / 2 + (int)blockIdx.y * s, xk = s / 2 + (int)blockIdx.x * s;
    const int z0 = max(0, zk - s), z1 = min(nz, zk + s + 1);
    const int x0 = max(0, xk - s), x1 = min(nx, xk + s + 1);
    const int WZ = z1 - z0, WX = x1 - x0;
    const int PZ = WZ + 2 * h, PX = WX + 2 * h;
    double *G = reinterpret_cast<double *>(smem);   // [n][n]
    double *rhs = G + n * n;                        // [n]
    double *red = rhs + n;                          // [2]: trace, pivot status
    double *RS = red + 2;                           // [nrs warps][PZ][2h + 1] row sums of one lag
    float *P = reinterpret_cast<float *>(RS + (size_t)nrs * PZ * (2 * h + 1));   // [PZ][PX]
    const long long plane = (long long)nz * nx;
    const float *m2 = mrem + param * plane;
    const float *m1 = mref + param * plane;
    const int t = threadIdx.x;

    for (int i = t; i < PZ * PX; i += blockDim.x) {
        int pz = i / PX, px = i - pz * PX;
        int z = z0 - h + pz, x = x0 - h + px;
        P[i] = (z >= 0 && z < nz && x >= 0 && x < nx) ? m2[(long long)z * nx + x] : 0.f;
    }
    if (t == 0) {
        red[0] = 0.0;
        red[1] = 0.0;
    }
    __syncthreads();

    // A[p, u] = m''(p - (a, b)) = P[pz + oz_u][px + ox_u], u = (a + h) flen + (b + h),
    // origin (oz_u, ox_u) = (2h - u / flen, 2h - u % flen) in [0, 2h]^2
    {
        const int warp = t >> 5, lane = t & 31, W2 = 2 * h + 1;
        double *rs = RS + (size_t)warp * PZ * W2;
        const int nlag = 2 * h * (4 * h + 1) + (2 * h + 1);   // dz > 0, or dz = 0 and dx >= 0
        for (int li = warp; li < nlag && warp < nrs; li += nrs) {
            const int dz = li < 2 * h + 1 ? 0 : 1 + (li - (2 * h + 1)) / (4 * h + 1);
            const int dx = li < 2 * h + 1 ? li : (li - (2 * h + 1)) % (4 * h + 1) - 2 * h;
            const int oz0 = max(0, -dz), oz1 = min(2 * h, 2 * h - dz);   // origins of u with u + d a tap
            const int ox0 = max(0, -dx), ox1 = min(2 * h, 2 * h - dx);
            // rs[r][ox] = sum_{c = ox}^{ox + WX - 1} P[r][c] P[r + dz][c + dx]
            for (int r = oz0 + lane; r < oz1 + WZ; r += 32) {
                const float *a = P + r * PX, *b = P + (r + dz) * PX + dx;
                double acc = 0.0;
                for (int c = ox0; c < ox0 + WX; ++c) acc = fma((double)a[c], (double)b[c], acc);
                rs[r * W2 + ox0] = acc;
                for (int ox = ox0 + 1; ox <= ox1; ++ox) {
                    acc = fma((double)a[ox + WX - 1], (double)b[ox + WX - 1], acc);
                    acc = fma(-(double)a[ox - 1], (double)b[ox - 1], acc);
                    rs[r * W2 + ox] = acc;
                }
            }
            __syncwarp();
            // S(oz, ox) = sum_{r = oz}^{oz + WZ - 1} rs[r][ox] -> G[u][v] and G[v][u]
            for (int ox = ox0 + lane; ox <= ox1; ox += 32) {
                double acc = 0.0;
                for (int r = oz0; r < oz0 + WZ; ++r) acc += rs[r * W2 + ox];
                for (int oz = oz0; oz <= oz1; ++oz) {
                    if (oz > oz0) acc += rs[(oz + WZ - 1) * W2 + ox] - rs[(oz - 1) * W2 + ox];
                    const int u = (2 * h - oz) * flen + (2 * h - ox);
                    const int v = (2 * h - oz - dz) * flen + (2 * h - ox - dx);
                    G[u * n + v] = acc;
                    G[v * n + u] = acc;
                }
            }
            __syncwarp();
        }
    }
    for (int u = t; u < n; u += blockDim.x) {
        const int ozu = 2 * h - u / flen, oxu = 2 * h - u % flen;
        double acc = 0.0;
        for (int pz = 0; pz < WZ; ++pz) {
            const float *ru = P + (pz + ozu) * PX + oxu;
            const float *r1 = m1 + (long long)(z0 + pz) * nx + x0;
            for (int px = 0; px < WX; ++px) acc = fma((double)ru[px], (double)r1[px], acc);
        }
        rhs[u] = acc;
    }
    __syncthreads();
    if (t == 0) {
        double tr = 0.0;
        for (int u = 0; u < n; ++u) tr += G[u * n + u];
        red[0] = tr;
    }
    __syncthreads();
    const double tr = red[0];
    float *out = filt + (((long long)param * nkz + blockIdx.y) * nkx + blockIdx.x) * n;
    if (tr == 0.0) {   // all-zero remigrated window: zero filter
        for (int u = t; u < n; u += blockDim.x) out[u] = 0.f;
        return;
    }
    const double reg = eps * tr / n;
    for (int u = t; u < n; u += blockDim.x) G[u * n + u] += reg;
    __syncthreads();

    // Cholesky G = L L^T, L in the lower triangle
    for (int k = 0; k < n; ++k) {
        if (t == 0) {
            double d = G[k * n + k];
            if (!(d > 0.0)) {
                red[1] = 1.0;
                d = 1.0;
            }
            G[k * n + k] = sqrt(d);
        }
        __syncthreads();
        const double dk = G[k * n + k];
        for (int i = k + 1 + t; i < n; i += blockDim.x) G[i * n + k] /= dk;
        __syncthreads();
        const int m = n - k - 1;
        for (int e = t; e < m * m; e += blockDim.x) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j <= i) G[i * n + j] -= G[i * n + k] * G[j * n + k];
        }
        __syncthreads();
    }
    // L y = rhs, then L^T f = y (in place in rhs)
    for (int k = 0; k < n; ++k) {
        if (t == 0) rhs[k] /= G[k * n + k];
        __syncthreads();
        const double yk = rhs[k];
        for (int i = k + 1 + t; i < n; i += blockDim.x) rhs[i] -= G[i * n + k] * yk;
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {
        if (t == 0) rhs[k] /= G[k * n + k];
        __syncthreads();
        const double fk = rhs[k];
        for (int i = t; i < k; i += blockDim.x) rhs[i] -= G[k * n + i] * fk;
        __syncthreads();
    }
    const bool bad = red[1] != 0.0;
    if (bad && t == 0) atomicOr(flag, 1);
    for (int u = t; u < n; u += blockDim.x) out[u] = bad ? 0.f : (float)rhs[u];
}

__global__ void k_deblur_apply(const float *mref, const float *filt, int nz, int nx, int s, int flen, int nkz,
                               int nkx, float *out)
{
    const long long plane = (long long)nz * nx;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= plane) return;
    const int param = blockIdx.y;
    const int z = (int)(i / nx), x = (int)(i - (long long)(i / nx) * nx);
    const int n = flen * flen, h = flen / 2;
    const float *m1 = mref + param * plane;
    // covering nodes: the nearest node at or above, and the next one, per axis
    int kz[2], kx[2];
    float wz[2], wx[2];
    const int iz = z >= s / 2 ? (z - s / 2) / s : -1, ix = x >= s / 2 ? (x - s / 2) / s : -1;
    for (int q = 0; q < 2; ++q) {
        kz[q] = iz + q;
        kx[q] = ix + q;
        wz[q] = (kz[q] >= 0 && kz[q] < nkz) ? fmaxf(0.f, 1.f - fabsf((float)(z - (s / 2 + kz[q] * s))) / s) : 0.f;
        wx[q] = (kx[q] >= 0 && kx[q] < nkx) ? fmaxf(0.f, 1.f - fabsf((float)(x - (s / 2 + kx[q] * s))) / s) : 0.f;
    }
    const float *fk[4];
    float w[4];
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    float den = 0.f;
    for (int q = 0; q < 4; ++q) {
        const int a = q >> 1, b = q & 1;
        w[q] = wz[a] * wx[b];
        fk[q] = w[q] > 0.f ? filt + (((long long)param * nkz + kz[a]) * nkx + kx[b]) * n : nullptr;
        den += w[q];
    }
    for (int a = -h; a <= h; ++a) {
        const int zz = z - a;
        if (zz < 0 || zz >= nz) continue;
        for (int b = -h; b <= h; ++b) {
            const int xx = x - b;
            if (xx < 0 || xx >= nx) continue;
            const float v = m1[(long long)zz * nx + xx];
            const int u = (a + h) * flen + (b + h);
            for (int q = 0; q < 4; ++q)
                if (fk[q]) acc[q] = fmaf(fk[q][u], v, acc[q]);
        }
    }
    float num = 0.f;
    for (int q = 0; q < 4; ++q) num = fmaf(w[q], acc[q], num);
    out[param * plane + i] = den > 0.f ? num / den : 0.f;
}

// ---------------------------------------------------------------------------
// Nonstationary Wiener filter (App. E, Fourier form). Per comb node a block of
// N x N = 2s x 2s pixels (z_k - s .. z_k + s - 1, the same in x; zero outside
// the image). With A = F m'' and B = F m_rtm (F the N x N DFT) the block's
// result is Re F^-1 [conj(A) B / (|A|^2 + eps_k) B], eps_k = eps mean|A|^2
// (zero when m'' is zero), and the blocks are blended with the bilinear
// valence of the space-domain filters.
//
// k_wiener_block: one CTA per (node, plane); the block, its spectra and a
// transform buffer sit in shared memory as complex FP32; each 2D DFT runs
// along the rows, then the columns, each as one Cooley-Tukey split N = N1 N2
// (dft2) with a twiddle table; the block result goes to
// blk[plane][node][N*N].
// k_wiener_blend: one thread per pixel, the (up to) four covering blocks.
// ---------------------------------------------------------------------------
constexpr int kWienerThreads = 256, kWienerMaxS = 32;

// One Cooley-Tukey split of a length-N DFT, N = N1 N2 (N1 the divisor of N
// nearest sqrt N; 5 x 8 for N = 40): with n = N2 n1 + n2 and k = k1 + N1 k2,
//   X[k] = sum_n2 w^(N1 n2 k2) [ w^(n2 k1) sum_n1 x[N2 n1 + n2] w^(N2 n1 k1) ],
// w = exp(-+2 pi i / N): N1 + N2 terms per output instead of N. Pass A (the
// inner sums and the twiddle) writes tmp[row][n2 N1 + k1]; pass B the outputs.
// Applied to every row (stride 1 along a row, rows `rs` apart) or every
// column (stride N, columns 1 apart) of an N x N block.
__device__ int dft_split(int N)
{
    int best = 1;
    for (int d = 2; d <= N; ++d)
        if (N % d == 0 && fabsf((float)d * d - (float)N) < fabsf((float)best * best - (float)N)) best = d;
    return best;
}

__device__ void dft_pass_a(const float2 *src, float2 *tmp, const float2 *tw, int N, int N1, bool inverse, bool cols)
{
    const int N2 = N / N1, NN = N * N;
    for (int idx = threadIdx.x; idx < NN; idx += blockDim.x) {
        const int line = idx / N, e = idx - line * N;   // e = n2 N1 + k1
        const int n2 = e / N1, k1 = e - n2 * N1;
        const int st = cols ? N : 1, base = cols ? line : line * N;
        float re = 0.f, im = 0.f;
        int j = 0;
        for (int n1 = 0; n1 < N1; ++n1) {
            const float2 w = tw[j];
            const float wi = inverse ? w.y : -w.y;
            const float2 v = src[base + (N2 * n1 + n2) * st];
            re = fmaf(v.x, w.x, fmaf(-v.y, wi, re));
            im = fmaf(v.x, wi, fmaf(v.y, w.x, im));
            j += N2 * k1;
            while (j >= N) j -= N;
        }
        int jt = n2 * k1;
        while (jt >= N) jt -= N;
        const float2 w = tw[jt];
        const float wi = inverse ? w.y : -w.y;
        tmp[idx] = make_float2(re * w.x - im * wi, re * wi + im * w.x);
    }
    __syncthreads();
}

__device__ void dft_pass_b(const float2 *tmp, float2 *dst, const float2 *tw, int N, int N1, bool inverse, bool cols)
{
    const int N2 = N / N1, NN = N * N;
    for (int idx = threadIdx.x; idx < NN; idx += blockDim.x) {
        const int line = idx / N, k = idx - line * N;   // k = k1 + N1 k2
        const int k2 = k / N1, k1 = k - k2 * N1;
        float re = 0.f, im = 0.f;
        int j = 0;
        for (int n2 = 0; n2 < N2; ++n2) {
            const float2 w = tw[j];
            const float wi = inverse ? w.y : -w.y;
            const float2 v = tmp[line * N + n2 * N1 + k1];
            re = fmaf(v.x, w.x, fmaf(-v.y, wi, re));
            im = fmaf(v.x, wi, fmaf(v.y, w.x, im));
            j += N1 * k2;
            while (j >= N) j -= N;
        }
        dst[cols ? k * N + line : line * N + k] = make_float2(re, im);
    }
    __syncthreads();
}

// dst = DFT2(src) (sign -1) or the unscaled inverse (sign +1), rows then
// columns, via tmp (src is kept; dst and tmp are overwritten).
__device__ void dft2(const float2 *src, float2 *tmp, float2 *dst, const float2 *tw, int N, bool inverse)
{
    const int N1 = dft_split(N);
    dft_pass_a(src, tmp, tw, N, N1, inverse, false);
    dft_pass_b(tmp, dst, tw, N, N1, inverse, false);
    dft_pass_a(dst, tmp, tw, N, N1, inverse, true);
    dft_pass_b(tmp, dst, tw, N, N1, inverse, true);
}

__device__ void load_block(const float *g, int nz, int nx, int zc, int xc, int N, float2 *dst)
{
    const int s = N / 2;
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
        const int a = idx / N, b = idx - a * N;
        const int z = zc - s + a, x = xc - s + b;
        const float v = (z >= 0 && z < nz && x >= 0 && x < nx) ? g[(long long)z * nx + x] : 0.f;
        dst[idx] = make_float2(v, 0.f);
    }
}

__global__ void __launch_bounds__(kWienerThreads) k_wiener_block(const float *mref, const float *mrem, int nz, int nx,
                                                                 int s, int nkx, float eps, float *blk)
{
    extern __shared__ __align__(16) float2 wsm[];
    const int N = 2 * s, NN = N * N;
    float2 *tw = wsm;            // [N] (cos, sin)(2 pi k / N)
    float2 *P = tw + N;          // [NN] input / product
    float2 *Q = P + NN;          // [NN] transform buffer
    float2 *A = Q + NN;          // [NN] F m''
    float2 *B = A + NN;          // [NN] F m_rtm
    __shared__ float red[kWienerThreads / 32];
    const int node = blockIdx.x, plane = blockIdx.y;
    const int kz = node / nkx, kx = node - kz * nkx;
    const int zc = s / 2 + kz * s, xc = s / 2 + kx * s;
    const long long pl = (long long)nz * nx;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        float sn, cs;
        sincospif(2.f * (float)k / (float)N, &sn, &cs);
        tw[k] = make_float2(cs, sn);
    }
    load_block(mrem + plane * pl, nz, nx, zc, xc, N, P);
    __syncthreads();
    dft2(P, Q, A, tw, N, false);
    load_block(mref + plane * pl, nz, nx, zc, xc, N, P);
    __syncthreads();
    dft2(P, Q, B, tw, N, false);
    // eps_k = eps * mean |A|^2
    float pw = 0.f;
    for (int idx = threadIdx.x; idx < NN; idx += blockDim.x) pw = fmaf(A[idx].x, A[idx].x, fmaf(A[idx].y, A[idx].y, pw));
    for (int o = 16; o > 0; o >>= 1) pw += __shfl_xor_sync(0xffffffffu, pw, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = pw;
    __syncthreads();
    float tot = 0.f;
    for (int w = 0; w < kWienerThreads / 32; ++w) tot += red[w];
    const float eps_k = eps * tot / (float)NN;
    // P = Lam^-1 B = conj(A) B B / (|A|^2 + eps_k)
    for (int idx = threadIdx.x; idx < NN; idx += blockDim.x) {
        float2 r = make_float2(0.f, 0.f);
        if (tot > 0.f) {
            const float2 a = A[idx], b = B[idx];
            const float den = fmaf(a.x, a.x, fmaf(a.y, a.y, eps_k));
            const float2 l = make_float2((a.x * b.x + a.y * b.y) / den, (a.x * b.y - a.y * b.x) / den);   // conj(a) b / den
            r = make_float2(l.x * b.x - l.y * b.y, l.x * b.y + l.y * b.x);
        }
        P[idx] = r;
    }
    __syncthreads();
    dft2(P, Q, A, tw, N, true);
    float *out = blk + ((long long)plane * gridDim.x + node) * NN;
    const float scale = 1.f / (float)NN;
    for (int idx = threadIdx.x; idx < NN; idx += blockDim.x) out[idx] = A[idx].x * scale;
}

__global__ void k_wiener_blend(const float *blk, int nz, int nx, int s, int nkz, int nkx, float *out)
{
    const long long plane = (long long)nz * nx;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= plane) return;
    const int param = blockIdx.y;
    const int z = (int)(i / nx), x = (int)(i - (long long)(i / nx) * nx);
    const int N = 2 * s, NN = N * N;
    const int iz = z >= s / 2 ? (z - s / 2) / s : -1, ix = x >= s / 2 ? (x - s / 2) / s : -1;
    float num = 0.f, den = 0.f;
    for (int a = 0; a < 2; ++a) {
        const int kz = iz + a;
        if (kz < 0 || kz >= nkz) continue;
        const int dz = z - (s / 2 + kz * s);
        const float wz = fmaxf(0.f, 1.f - fabsf((float)dz) / s);
        for (int b = 0; b < 2; ++b) {
            const int kx = ix + b;
            if (kx < 0 || kx >= nkx) continue;
            const int dx = x - (s / 2 + kx * s);
            const float w = wz * fmaxf(0.f, 1.f - fabsf((float)dx) / s);
            if (w <= 0.f) continue;
            num = fmaf(w, blk[(((long long)param * nkz + kz) * nkx + kx) * NN + (dz + s) * N + (dx + s)], num);
            den += w;
        }
    }
    out[param * plane + i] = den > 0.f ? num / den : 0.f;
}

}  // namespace

int wiener_max_spacing() { return kWienerMaxS; }

size_t wiener_smem(int s)
{
    const size_t N = 2 * (size_t)s;
    return (N + 4 * N * N) * sizeof(float2);
}

cudaError_t launch_wiener(const float *mref, const float *mrem, int nz, int nx, int s, double eps, float *blk,
                          float *out, cudaStream_t st)
{
    const int nkz = deblur_nodes(nz, s), nkx = deblur_nodes(nx, s);
    const size_t sm = wiener_smem(s);
    cudaError_t e = cudaFuncSetAttribute(k_wiener_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_wiener_block<<<dim3(nkz * nkx, 2), kWienerThreads, sm, st>>>(mref, mrem, nz, nx, s, nkx, (float)eps, blk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long plane = (long long)nz * nx;
    k_wiener_blend<<<dim3((unsigned)((plane + 255) / 256), 2), 256, 0, st>>>(blk, nz, nx, s, nkz, nkx, out);
    return cudaGetLastError();
}

// Shared memory of k_deblur_solve with nrs warps forming lag sums.
size_t deblur_solve_smem(int nz, int nx, int s, int flen, int nrs)
{
    const int n = flen * flen, h = flen / 2;
    const int wz = std::min(nz, 2 * s + 1), wx = std::min(nx, 2 * s + 1);
    return ((size_t)n * n + n + 2 + (size_t)nrs * (wz + 2 * h) * (2 * h + 1)) * sizeof(double) +
           (size_t)(wz + 2 * h) * (wx + 2 * h) * sizeof(float);
}

// Warps of k_deblur_solve that form lag sums: as many as fit (at most all),
// 0 if not even one does.
int deblur_solve_warps(int nz, int nx, int s, int flen)
{
    int nrs = kSolveThreads / 32;
    while (nrs > 0 && deblur_solve_smem(nz, nx, s, flen, nrs) > kDeblurSmemLimit) --nrs;
    return nrs;
}

int deblur_nodes(int n, int s) { return n > s / 2 ? (n - 1 - s / 2) / s + 1 : 0; }

cudaError_t launch_deblur(const float *mref, const float *mrem, int nz, int nx, int s, int flen, double eps,
                          float *filt, float *out, int *flag, cudaStream_t st)
{
    const int nkz = deblur_nodes(nz, s), nkx = deblur_nodes(nx, s);
    const int nrs = deblur_solve_warps(nz, nx, s, flen);
    if (nrs < 1) return cudaErrorInvalidValue;
    const size_t sm = deblur_solve_smem(nz, nx, s, flen, nrs);
    cudaError_t e = cudaFuncSetAttribute(k_deblur_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_deblur_solve<<<dim3(nkx, nkz, 2), kSolveThreads, sm, st>>>(mref, mrem, nz, nx, s, flen, eps, filt, flag, nrs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long plane = (long long)nz * nx;
    k_deblur_apply<<<dim3((unsigned)((plane + 255) / 256), 2), 256, 0, st>>>(mref, filt, nz, nx, s, flen, nkz, nkx,
                                                                              out);
    return cudaGetLastError();
}

}  // namespace lsrtm
