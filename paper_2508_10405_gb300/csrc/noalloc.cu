// Born modelling for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: plugins whose host application owns
// the GPU memory pool and forbids foreign allocations, and real-time loops
// where an allocation (and the implicit device synchronisation it can cause)
// is not allowed. lsrtm_born_static serves them: it computes the same d = L dm
// as lsrtm_born, but every byte of device workspace it needs comes from one
// file-scope __device__ array of fixed size (kStaticBytes), which every GPU
// that loads this library holds until the process exits. The caller passes
// the model, wavelet, perturbation and output as device pointers and the
// geometry as host arrays, which are copied into the array with
// cudaMemcpyAsync before the call returns (the caller may free them
// afterwards); the call allocates nothing on the device (no cudaMalloc, no
// cudaFree, no allocating library routine). Inputs are not checked for
// finiteness: a NaN or Inf in the model gives non-finite records rather than
// an error status.
//
// Shared-state rules:
//   * the array is shared by every call on a device and keeps the contents of
//     the last call; each call re-initialises everything it reads (model,
//     profiles, receiver tables) and zeroes the wavefields before use;
//   * calls whose GPU work overlaps (different streams, or different host
//     threads on one device without ordering) race on the array: order them;
//   * the first call on a device looks up the device address of the array
//     (cudaGetSymbolAddress) and configures the kernels; make that first call
//     before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/lsrtm.h"
#include "lsrtm_internal.cuh"

namespace lsrtm {

void set_last_error(const std::string &msg);

namespace {

constexpr size_t kStaticBytes = 32ull << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

void *g_ws_addr[kMaxDevices];
std::mutex g_ws_mutex;

lsrtm_status fail(lsrtm_status st, const std::string &msg)
{
    set_last_error(msg);
    return st;
}

// Device address of g_static_ws on the current device (looked up once per device).
lsrtm_status static_workspace(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LSRTM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(LSRTM_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_ws_mutex);
    if (!g_ws_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess || !p)
            return fail(LSRTM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        e = ensure_kernels_configured();
        if (e != cudaSuccess)
            return fail(LSRTM_ERR_CUDA, std::string("kernel configuration: ") + cudaGetErrorString(e));
        g_ws_addr[dev] = p;
    }
    *out = g_ws_addr[dev];
    return LSRTM_OK;
}

bool on_device(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// CPML coefficients (same profile as lsrtm_create) computed on the device:
// damping d0 r^2 and alpha = pi f0 (1 - r), r = distance beyond the
// interface half node / npml; zero at and inside the interface.
__global__ void k_cpml_static(int N, int o, int n, int npml, double h, double vmax, double f0, double dt,
                              float *ai, float *bi, float *ah, float *bh)
{
    const double pi = 3.14159265358979323846;
    double d0 = npml > 0 ? -3.0 * vmax * log(1e-4) / (2.0 * npml * h) : 0.0;
    double lo = o - 0.5, hi = o + n - 0.5;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        for (int half = 0; half < 2; ++half) {
            double pos = i + 0.5 * half;
            double dist = fmax(0.0, fmax(lo - pos, pos - hi));
            float a = 0.f, b = 0.f;
            if (dist > 0.0) {
                double r = dist / npml;
                double d = d0 * r * r;
                double al = pi * f0 * (1.0 - r);
                if (al < 0) al = 0;
                double bb = exp(-(d + al) * dt);
                b = (float)bb;
                a = (float)(d * (bb - 1.0) / (d + al));
            }
            if (half) {
                ah[i] = a;
                bh[i] = b;
            } else {
                ai[i] = a;
                bi[i] = b;
            }
        }
    }
}

// Source cells and receivers grouped per (shot, CTA tile) in CSR form; one
// thread, for the small problems the static workspace admits.
__global__ void k_geom_static(GridDev g, int nshot, int txo, int tzc, int ntx, int ntiles, const int *src_idx,
                              const int *rec_ptr, const int *rec_idx, int *src_cell, int *tptr, int *tcur,
                              int2 *trec)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    auto cell_of = [&](long long k) {
        long long ix = k % g.nx, t = k / g.nx, iy = t % g.ny, iz = t / g.ny;
        return (iz + g.z0) * g.rowz + (iy + g.y0) * g.pitch + (ix + g.x0);
    };
    auto tile_of = [&](long long c) {
        int z = (int)(c / g.rowz), x = (int)(c % g.pitch);
        return (z / tzc) * ntx + x / txo;
    };
    const int nt = nshot * ntiles;
    for (int i = 0; i <= nt; ++i) tptr[i] = 0;
    for (int s = 0; s < nshot; ++s) {
        src_cell[s] = (int)cell_of(src_idx[s]);
        for (int r = rec_ptr[s]; r < rec_ptr[s + 1]; ++r) tptr[s * ntiles + tile_of(cell_of(rec_idx[r])) + 1]++;
    }
    for (int i = 0; i < nt; ++i) {
        tptr[i + 1] += tptr[i];
        tcur[i] = tptr[i];
    }
    for (int s = 0; s < nshot; ++s)
        for (int r = rec_ptr[s]; r < rec_ptr[s + 1]; ++r) {
            long long c = cell_of(rec_idx[r]);
            trec[tcur[s * ntiles + tile_of(c)]++] = make_int2((int)c, r);
        }
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace lsrtm

using namespace lsrtm;

extern "C" lsrtm_status lsrtm_born_static(const lsrtm_config *cfg, const float *vp, const float *rho,
                                          const float *wavelet, const lsrtm_geometry *geom, const float *dm,
                                          float *d, void *stream)
{
    set_last_error("");
    if (!cfg || !vp || !rho || !wavelet || !geom || !dm || !d) return fail(LSRTM_ERR_ARG, "null argument");
    if (cfg->ndim != 2) return fail(LSRTM_ERR_ARG, "lsrtm_born_static supports 2D grids only");
    if (cfg->fd_order != 4 && cfg->fd_order != 8) return fail(LSRTM_ERR_ARG, "fd_order must be 4 or 8");
    if (cfg->nz < 1 || cfg->nx < 1 || cfg->nt < 1) return fail(LSRTM_ERR_ARG, "empty grid or nt < 1");
    if (cfg->npml < cfg->fd_order / 2) return fail(LSRTM_ERR_ARG, "npml must be >= fd_order/2");
    if (!(cfg->dt > 0) || !(cfg->dx > 0) || !(cfg->dz > 0)) return fail(LSRTM_ERR_ARG, "non-positive spacing or dt");
    if (!(cfg->pml_vmax > 0))
        return fail(LSRTM_ERR_ARG, "lsrtm_born_static needs cfg->pml_vmax > 0 (the maximum velocity)");
    if (!on_device(vp) || !on_device(rho) || !on_device(wavelet) || !on_device(dm) || !on_device(d))
        return fail(LSRTM_ERR_ARG, "lsrtm_born_static takes device pointers only");
    const int M = cfg->fd_order / 2;
    double c[4];
    if (M == 2) {
        c[0] = 9.0 / 8.0;
        c[1] = -1.0 / 24.0;
    } else {
        c[0] = 1225.0 / 1024.0;
        c[1] = -245.0 / 3072.0;
        c[2] = 49.0 / 5120.0;
        c[3] = -5.0 / 7168.0;
    }
    {
        double s = 0.0, inv2 = 1.0 / (cfg->dz * cfg->dz) + 1.0 / (cfg->dx * cfg->dx);
        for (int l = 0; l < M; ++l) s += std::fabs(c[l]);
        if (!(cfg->dt < 1.0 / (cfg->pml_vmax * std::sqrt(inv2) * s)))
            return fail(LSRTM_ERR_CFL, "dt exceeds the stability limit");
    }
    // grid description, as lsrtm_create lays it out
    GridDev g{};
    g.ndim = 2;
    g.M = M;
    g.nz = cfg->nz;
    g.ny = 1;
    g.nx = cfg->nx;
    g.z0 = cfg->npml;
    g.y0 = 0;
    g.x0 = cfg->npml;
    g.Nz = g.nz + 2 * cfg->npml;
    g.Ny = 1;
    g.Nx = g.nx + 2 * cfg->npml;
    g.pitch = (g.Nx + 31) / 32 * 32;
    g.rowz = g.pitch;
    g.plane = (long long)g.Nz * g.pitch;
    g.dt = (float)cfg->dt;
    g.nt = cfg->nt;
    for (int l = 0; l < kMaxM; ++l) {
        double cl = l < M ? c[l] : 0.0;
        g.cz[l] = (float)(cl / cfg->dz);
        g.cy[l] = 0.f;
        g.cx[l] = (float)(cl / cfg->dx);
    }
    const long long nint = (long long)g.nz * g.nx;
    // geometry checks (host arrays)
    if (geom->nshot < 1 || !geom->src_idx || !geom->rec_ptr) return fail(LSRTM_ERR_ARG, "invalid geometry");
    if (geom->win_x0 || geom->win_nx) return fail(LSRTM_ERR_ARG, "lsrtm_born_static does not take aperture windows");
    const int nshot = geom->nshot;
    if (geom->rec_ptr[0] != 0) return fail(LSRTM_ERR_GEOMETRY, "rec_ptr[0] must be 0");
    for (int s = 0; s < nshot; ++s) {
        if (geom->rec_ptr[s + 1] < geom->rec_ptr[s]) return fail(LSRTM_ERR_GEOMETRY, "rec_ptr not monotone");
        if (geom->src_idx[s] < 0 || geom->src_idx[s] >= nint)
            return fail(LSRTM_ERR_GEOMETRY, "source outside the interior grid");
    }
    const long long nrec = geom->rec_ptr[nshot];
    if (nrec > 0 && !geom->rec_idx) return fail(LSRTM_ERR_ARG, "invalid geometry");
    for (long long r = 0; r < nrec; ++r)
        if (geom->rec_idx[r] < 0 || geom->rec_idx[r] >= nint)
            return fail(LSRTM_ERR_GEOMETRY, "receiver outside the interior grid");
    const int txo = march2d_txo(M);
    const int nchunk = (g.Nz + 56) / 112 > 1 ? (g.Nz + 56) / 112 : 1;
    const int tzc = (g.Nz + nchunk - 1) / nchunk;
    const int ntx = (g.Nx + txo - 1) / txo, ntz = (g.Nz + tzc - 1) / tzc;
    const int ntiles = ntx * ntz;

    // carve the static workspace
    const size_t P = (size_t)g.plane;
    size_t off[16], sz[16];
    sz[0] = P * 4;                          // kdt
    sz[1] = P * 4;                          // binv
    sz[2] = P * 8;                          // kd2
    sz[3] = P * 8;                          // br2
    sz[4] = 4 * ((size_t)g.Nz + 1 + g.Nx) * 4;   // CPML profiles
    sz[5] = (size_t)nshot * 4;              // src_idx copy
    sz[6] = (size_t)(nshot + 1) * 4;        // rec_ptr copy
    sz[7] = (size_t)(nrec > 0 ? nrec : 1) * 4;   // rec_idx copy
    sz[8] = (size_t)nshot * 4;              // src_cell
    sz[9] = ((size_t)nshot * ntiles + 1) * 4;    // tile receiver offsets
    sz[10] = (size_t)nshot * ntiles * 4;    // tile cursors
    sz[11] = (size_t)(nrec > 0 ? nrec : 1) * 8;  // tile receivers
    sz[12] = 10 * P * 4;                    // wavefield ping
    sz[13] = 10 * P * 4;                    // wavefield pong
    sz[14] = 4 * P * 4;                     // node CPML memories
    size_t total = 0;
    for (int i = 0; i < 15; ++i) {
        off[i] = total;
        total += align256(sz[i]);
    }
    if (total > kStaticBytes) {
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "problem needs %zu bytes of workspace; lsrtm_born_static has a fixed %zu-byte static "
                      "workspace (use lsrtm_create/lsrtm_born for larger problems)",
                      total, (size_t)kStaticBytes);
        return fail(LSRTM_ERR_OOM, buf);
    }
    void *base = nullptr;
    lsrtm_status st = static_workspace(&base);
    if (st != LSRTM_OK) return st;
    auto at = [&](int i) { return static_cast<unsigned char *>(base) + off[i]; };
    cudaStream_t s = static_cast<cudaStream_t>(stream);

#define SCU(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(LSRTM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

    float *kdt = reinterpret_cast<float *>(at(0));
    float *binv = reinterpret_cast<float *>(at(1));
    float2 *kd2 = reinterpret_cast<float2 *>(at(2));
    float2 *br2 = reinterpret_cast<float2 *>(at(3));
    float *prof = reinterpret_cast<float *>(at(4));
    int *src_copy = reinterpret_cast<int *>(at(5));
    int *rp_copy = reinterpret_cast<int *>(at(6));
    int *ri_copy = reinterpret_cast<int *>(at(7));
    int *src_cell = reinterpret_cast<int *>(at(8));
    int *tptr = reinterpret_cast<int *>(at(9));
    int *tcur = reinterpret_cast<int *>(at(10));
    int2 *trec = reinterpret_cast<int2 *>(at(11));
    float *st0 = reinterpret_cast<float *>(at(12));
    float *st1 = reinterpret_cast<float *>(at(13));
    float *psiv = reinterpret_cast<float *>(at(14));

    // model, perturbation and profiles
    SCU(cudaMemsetAsync(kdt, 0, sz[0], s));
    SCU(cudaMemsetAsync(binv, 0, sz[1], s));
    SCU(launch_model_prep(g, vp, rho, kdt, binv, s));
    SCU(launch_pert_prep(g, dm, kdt, binv, kd2, br2, s));
    Pml pml{};
    {
        const int N[3] = {g.Nz, 1, g.Nx};
        const int o[3] = {g.z0, 0, g.x0};
        const int ni[3] = {g.nz, 1, g.nx};
        const double hh[3] = {cfg->dz, 1.0, cfg->dx};
        size_t po = 0;
        SCU(cudaMemsetAsync(prof, 0, sz[4], s));
        for (int dd = 0; dd < 3; ++dd) {
            float *b = prof + po;
            if (dd != 1)
                k_cpml_static<<<(N[dd] + 255) / 256, 256, 0, s>>>(N[dd], o[dd], ni[dd], cfg->npml, hh[dd],
                                                                  cfg->pml_vmax, cfg->f0, cfg->dt, b, b + N[dd],
                                                                  b + 2 * N[dd], b + 3 * N[dd]);
            SCU(cudaGetLastError());
            pml.ai[dd] = b;
            pml.bi[dd] = b + N[dd];
            pml.ah[dd] = b + 2 * N[dd];
            pml.bh[dd] = b + 3 * N[dd];
            po += 4 * (size_t)N[dd];
        }
    }
    // geometry tables
    SCU(cudaMemcpyAsync(src_copy, geom->src_idx, sz[5], cudaMemcpyHostToDevice, s));
    SCU(cudaMemcpyAsync(rp_copy, geom->rec_ptr, sz[6], cudaMemcpyHostToDevice, s));
    if (nrec > 0) SCU(cudaMemcpyAsync(ri_copy, geom->rec_idx, (size_t)nrec * 4, cudaMemcpyHostToDevice, s));
    k_geom_static<<<1, 1, 0, s>>>(g, nshot, txo, tzc, ntx, ntiles, src_copy, rp_copy, ri_copy, src_cell, tptr,
                                  tcur, trec);
    SCU(cudaGetLastError());

    // time loop, one shot at a time through one wavefield slot
    Step2D a{};
    a.g = g;
    a.pml = pml;
    a.kdt = kdt;
    a.binv = binv;
    a.kd2 = kd2;
    a.br2 = br2;
    a.psiv = psiv;
    a.sstride = 10 * g.plane;
    a.vstride = 4 * g.plane;
    a.tzc = tzc;
    a.wav = wavelet;
    a.wav_per_shot = cfg->wavelet_per_shot;
    a.src_cell = src_cell;
    a.src_scale = (float)(cfg->dt / (cfg->dz * cfg->dx));
    a.trec.ptr = tptr;
    a.trec.rec = trec;
    a.trec.ntiles = ntiles;
    a.dstage = d;   // records go straight to the caller's output
    for (int shot = 0; shot < nshot; ++shot) {
        SCU(cudaMemsetAsync(st0, 0, sz[12], s));
        SCU(cudaMemsetAsync(st1, 0, sz[13], s));
        SCU(cudaMemsetAsync(psiv, 0, sz[14], s));
        a.shot0 = shot;
        for (int n = 0; n < g.nt; ++n) {
            a.n = n;
            a.in = (n & 1) ? st1 : st0;
            a.out = (n & 1) ? st0 : st1;
            SCU(launch_fwd2d(a, 1, true, false, false, s));
        }
    }
#undef SCU
    return LSRTM_OK;
}
