// Host engine and C ABI of the LSRTM operator library (see include/lsrtm.h).
//
// The engine validates the configuration, lays the padded model and the
// per-shot wavefield slots out in HBM, groups shots into batches that one
// launch advances together, captures each batch's nt-step loop in a CUDA
// graph, caches the background boundary bands across L^T calls, and runs
// the CGNR driver with FP64 device scalars. All device work runs on a private
// stream ordered after and before the caller's stream by events.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lsrtm.h"
#include "lsrtm_internal.cuh"
#include "wiener.cuh"
#include "psfhess3d.cuh"

using namespace lsrtm;

namespace {

thread_local std::string g_last_error;

lsrtm_status fail(lsrtm_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(LSRTM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CHECK(expr)                            \
    do {                                       \
        lsrtm_status s_ = (expr);              \
        if (s_ != LSRTM_OK) return s_;         \
    } while (0)

// Planes per wavefield slot: 10 ping-pong planes (Born: (p, dp) (vx, dvx)
// (vz, dvz) (psi_px, dpsi_px) (psi_pz, dpsi_pz) as float2 pairs; background
// only: p vx vz psi_px psi_pz; adjoint: (p, lambda_p) (vx, lambda_vx)
// (vz, lambda_vz) pairs and four lambda CPML memories), 4 in-place node CPML
// planes (forward).
constexpr int kStatePlanes2D = 10;
constexpr int kPsivPlanes2D = 4;
constexpr int kStatePlanes3D = 20;

enum GraphKind { G_BORN = 0, G_BG = 1, G_BG_HESS = 2, G_ADJ = 3, G_MODEL = 6 };

}  // namespace

struct lsrtm_handle {
    lsrtm_config cfg{};
    GridDev g{};                 // grid of the wavefield slots (the widest aperture window)
    GridDev gm{};                // grid of the model and the images
    // per-shot aperture windows (2D)
    bool win = false;
    int *win_x0_d = nullptr, *win_nx_d = nullptr;
    std::vector<int> win_x0_h, win_nx_h;
    cudaStream_t user = nullptr;
    cudaStream_t work = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int nshot = 0;
    long long nrec_total = 0;
    long long nint = 0;
    std::vector<int> rec_ptr;
    std::vector<double> rec_off_h;   // horizontal source-receiver offset of every receiver row (m)
    int *mute_n0 = nullptr;          // muting: per receiver the first sample after the mute time
    float *mute_a0 = nullptr;        // muting: per receiver (t_n0 - mute time) / taper
    float *mute_fo = nullptr;        // muting: per receiver the far-offset factor
    float *dstage2 = nullptr;        // second [nrec_total][nt] stage (host inputs of the muting)
    // device model and geometry
    float *kdt = nullptr, *binv = nullptr;
    float2 *kd2 = nullptr, *br2 = nullptr;   // (dt kappa, perturbation) and (1/rho, perturbation)
    float *pml_buf = nullptr;
    Pml pml{};
    float *wav = nullptr;
    int *src_cell = nullptr;
    int *trec_ptr = nullptr;
    size_t trec_ptr_cap = 0;
    std::vector<int2> rec_cells_h;   // 2D: per shot (rec_ptr ranges) the receiver cells and rows
    int2 *trec = nullptr;
    TileRecs trv{};
    float src_scale = 0.f;
    int txo = 0, tzc = 0;        // CTA output columns and z-chunk rows (2D)
    // 3D receiver maps: per shot and node, the first of its receivers in rcell/rrow
    int *rmap = nullptr, *rptr = nullptr, *rcell = nullptr, *rrow = nullptr;
    int fs_planes = 3;           // planes of the saved background final state per shot
    // wavefield slots
    int batch = 1;
    float *st[2] = {nullptr, nullptr};
    long long sstride = 0;
    long long sstride1 = 0;      // slot stride of st[1] (3D: the fused kernels' pong buffer)
    Step3F f3born[2];            // fused 3D Born step arguments reading st[0] / st[1]
    Adj3F f3adj[2];              // fused 3D adjoint step arguments reading st[0] / st[1]
    Maps2D m2d[2];             // 2D TMA row maps reading st[0] / st[1]
    bool tma2d = false;          // the 2D Born and migration kernels stage rows by TMA (no aperture windows)
    int *kerr = nullptr;         // device error words: [0] fused-kernel tile copies, [1] non-finite guard
    int guard_K = 0;             // time steps between non-finite guard checks (0: off)
    long long guard_count = 0;   // guard launches queued or captured so far
    std::map<std::pair<int, int>, long long> graph_guards;   // guard launches per captured graph
    int *poll_h = nullptr;       // pinned host copies of the error words, two per CG poll slot
    cudaEvent_t poll_ev[2] = {nullptr, nullptr};
    float *psiv = nullptr;
    long long vstride = 0;
    float2 *img = nullptr;
    double2 *img_acc = nullptr;
    float *hess = nullptr;
    double *hess_acc = nullptr;
    float *hess_img = nullptr;
    bool hess_ready = false;
    // background cache
    Bands bands{};
    void *band_mem = nullptr;
    float *final_state = nullptr;
    bool bg_cached = false;
    // checkpointed reconstruction (App. A alternative when the bands do not fit)
    bool ckpt = false;
    int ck_K = 0, ck_nseg = 0, ck_planes = 0;
    float *rec[2] = {nullptr, nullptr};   // background state for the recomputation
    float *rec_psiv = nullptr;
    void *ck_mem = nullptr;               // [nseg][batch][ck_planes][plane], FP32 or 16-bit
    int ck_fmt = BAND_F32;                // BandFmt of the checkpoints
    float *ck_amax = nullptr;             // 16-bit checkpoints: [nseg][batch][ck_planes] plane maxima
    Bands segbands{};                     // bands of one segment of one batch
    // staging
    float *dstage = nullptr;     // [nrec_total][nt]
    float *mstage = nullptr;     // [2][nint]
    float *gstage = nullptr;     // [2][nint]
    float *scratch1 = nullptr;   // [nint]
    float *db_filt = nullptr;    // deblurring filters, grown on demand
    size_t db_cap = 0;
    float *db_out = nullptr;     // [2][nint]
    float *wn_blk = nullptr;     // Wiener block results, grown on demand
    size_t wn_cap = 0;
    // interpolated PSF Hessian (App. D)
    float4 *ph_pt = nullptr;     // node windows, grown on demand
    size_t ph_cap = 0;
    float *ph_vec = nullptr;     // [8][2 nint]: x, r, s, p, q, staged input, staged PSFs (Vp, Ip)
    double *ph_scal = nullptr;   // [0] gamma [1] gamma_new [2] <q,q> [3] <d,d>
    double *ph_mis = nullptr;    // per-iteration <r,r>
    int ph_mis_cap = 0;
    // Krylov
    float *cg_x = nullptr, *cg_s = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_minv = nullptr;
    float *cg_r = nullptr;
    double *scal = nullptr;      // device scalars: [0] gamma [1] gamma_new [2] <q,q> [3] <d,d> [5] 1.0
    double *dotwork = nullptr;
    double *mis_dev = nullptr;   // per-iteration <r,r>
    int mis_cap = 0;
    float *fscal = nullptr;      // device float scalars
    int *flag = nullptr;
    // CGNR state
    bool cg_active = false;
    int cg_mask = 3, cg_precond = 0, cg_iter = 0;
    // event timing of the time loops (kind: 0 born, 1 background, 2 adjoint)
    bool timing = false;
    struct TimedLoop {
        int kind;
        cudaEvent_t a, b;
        long long launches;
        double cells;
    };
    std::vector<TimedLoop> pending;
    std::vector<cudaEvent_t> event_pool;
    double t_ms[3] = {0, 0, 0};
    long long t_launch[3] = {0, 0, 0};
    double t_cells[3] = {0, 0, 0};
    // graphs
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
    long long launches = 0;
    size_t bytes = 0;
    std::vector<void *> allocs;
};

namespace {

lsrtm_status dalloc(lsrtm_handle *h, void **p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (h->cfg.hbm_budget_bytes && h->bytes + bytes > h->cfg.hbm_budget_bytes)
        return fail(LSRTM_ERR_OOM, "workspace exceeds hbm_budget_bytes");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LSRTM_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->allocs.push_back(*p);
    h->bytes += bytes;
    cudaError_t e2 = cudaMemsetAsync(*p, 0, bytes, h->work);
    if (e2 != cudaSuccess) return fail(LSRTM_ERR_CUDA, cudaGetErrorString(e2));
    return LSRTM_OK;
}

template <class T>
lsrtm_status dalloc_t(lsrtm_handle *h, T **p, size_t count)
{
    return dalloc(h, reinterpret_cast<void **>(p), count * sizeof(T));
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Makes `src` usable on the device: returns it as is if it is device memory,
// else copies it into `stage` on the work stream.
lsrtm_status stage_in(lsrtm_handle *h, const float *src, float *stage, size_t count,
                      const float **dev)
{
    if (is_device_ptr(src)) {
        *dev = src;
        return LSRTM_OK;
    }
    CU(cudaMemcpyAsync(stage, src, count * sizeof(float), cudaMemcpyHostToDevice, h->work));
    *dev = stage;
    return LSRTM_OK;
}

lsrtm_status copy_out(lsrtm_handle *h, float *dst, const float *src, size_t count)
{
    CU(cudaMemcpyAsync(dst, src, count * sizeof(float), cudaMemcpyDefault, h->work));
    return LSRTM_OK;
}

// Orders the private work stream after everything queued on the caller's stream.
lsrtm_status begin_call(lsrtm_handle *h)
{
    g_last_error.clear();
    CU(cudaEventRecord(h->ev_in, h->user));
    CU(cudaStreamWaitEvent(h->work, h->ev_in, 0));
    return LSRTM_OK;
}

// Orders the caller's stream after the work queued by this call.
lsrtm_status check_kernel_error(lsrtm_handle *h);

lsrtm_status end_call(lsrtm_handle *h, bool sync)
{
    CU(cudaGetLastError());
    CU(cudaEventRecord(h->ev_out, h->work));
    CU(cudaStreamWaitEvent(h->user, h->ev_out, 0));
    if (sync) {
        CU(cudaStreamSynchronize(h->work));
        CHECK(check_kernel_error(h));
    }
    return LSRTM_OK;
}

// Staggered Taylor coefficients of order 2M (closed forms).
void fd_coeffs(int M, double *c)
{
    if (M == 2) {
        c[0] = 9.0 / 8.0;
        c[1] = -1.0 / 24.0;
    } else {
        c[0] = 1225.0 / 1024.0;
        c[1] = -245.0 / 3072.0;
        c[2] = 49.0 / 5120.0;
        c[3] = -5.0 / 7168.0;
    }
}

// CPML profile: damping d0 (r)^2, alpha = pi f0 (1 - r), r = distance beyond
// the interface half node / npml; zero (no memory) at and inside the interface.
void cpml_profile(int N, int o, int n, int npml, double h, double vmax, double f0, double dt,
                  float *ai, float *bi, float *ah, float *bh)
{
    const double pi = 3.14159265358979323846;
    double d0 = npml > 0 ? -3.0 * vmax * std::log(1e-4) / (2.0 * npml * h) : 0.0;
    auto coef = [&](double dist, float *a, float *b) {
        if (dist <= 0.0) {
            *a = 0.f;
            *b = 0.f;
            return;
        }
        double r = dist / npml;
        double d = d0 * r * r;
        double al = pi * f0 * (1.0 - r);
        if (al < 0) al = 0;
        double bb = std::exp(-(d + al) * dt);
        *b = (float)bb;
        *a = (float)(d * (bb - 1.0) / (d + al));
    };
    double lo = o - 0.5, hi = o + n - 0.5;
    for (int i = 0; i < N; ++i) {
        double di = std::max(0.0, std::max(lo - i, i - hi));
        double dh = std::max(0.0, std::max(lo - (i + 0.5), (i + 0.5) - hi));
        coef(di, &ai[i], &bi[i]);
        coef(dh, &ah[i], &bh[i]);
    }
}

Step2D step_args(lsrtm_handle *h, int shot0)
{
    Step2D a{};
    a.g = h->g;
    a.pml = h->pml;
    a.kdt = h->kdt;
    a.binv = h->binv;
    a.kd2 = h->kd2;
    a.br2 = h->br2;
    a.psiv = h->psiv;
    a.sstride = h->sstride;
    a.vstride = h->vstride;
    a.shot0 = shot0;
    a.wav = h->wav;
    a.wav_per_shot = h->cfg.wavelet_per_shot;
    a.src_cell = h->src_cell;
    a.src_scale = h->src_scale;
    a.trec = h->trv;
    a.dstage = h->dstage;
    a.bands = h->bands;
    a.hess = h->hess;
    a.img = h->img;
    a.tzc = h->tzc;
    a.win_nx = h->win ? h->win_nx_d : nullptr;
    a.pml_xstride = h->win ? h->g.Nx : 0;
    a.err = h->kerr;
    return a;
}

Step3D step3_args(lsrtm_handle *h, int shot0)
{
    Step3D a{};
    a.g = h->g;
    a.pml = h->pml;
    a.kdt = h->kdt;
    a.binv = h->binv;
    a.st = h->st[0];
    a.sstride = h->sstride;
    a.shot0 = shot0;
    a.wav = h->wav;
    a.wav_per_shot = h->cfg.wavelet_per_shot;
    a.src_cell = h->src_cell;
    a.src_scale = h->src_scale;
    a.bands = h->bands;
    a.hess = h->hess;
    a.dstage = h->dstage;
    a.rmap = h->rmap;
    a.rptr = h->rptr;
    a.rcell = h->rcell;
    a.rrow = h->rrow;
    return a;
}

bool is3d(const lsrtm_handle *h) { return h->g.ndim == 3; }

bool use_graphs(const lsrtm_handle *h) { return h->cfg.plan == LSRTM_PLAN_BATCHED; }

cudaEvent_t take_event(lsrtm_handle *h)
{
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

int timing_kind(int graph_kind)
{
    return graph_kind == G_BORN ? 0 : (graph_kind == G_ADJ ? 2 : 1);
}

// Kernel launches one nt-step loop of this kind contains (band-saving loops
// with 16-bit bands pack the bands after every step).
long long loop_launches(const lsrtm_handle *h, int kind)
{
    const long long nt = h->g.nt;
    const long long pack = (kind == G_BG || kind == G_BG_HESS) && h->bands.fmt != BAND_F32 ? nt : 0;
    if (h->g.ndim != 3 || kind == G_BORN || kind == G_ADJ) return nt + pack;   // 2D, fused 3D Born and adjoint
    return (kind == G_ADJ ? 2 * nt - 1 : 2 * nt) + pack;
}

template <class F>
lsrtm_status run_loop_n(lsrtm_handle *h, int kind, int tkind, int shot0, int bs, long long nlaunch,
                        long long nsteps, F &&body);

template <class F>
lsrtm_status run_loop(lsrtm_handle *h, int kind, int shot0, int bs, F &&body)
{
    return run_loop_n(h, kind, timing_kind(kind), shot0, bs, loop_launches(h, kind) + (h->win ? 1 : 0), h->g.nt,
                      body);
}

// Padded cells one time step of a batch advances (each windowed shot on its own grid).
double batch_cells(const lsrtm_handle *h, int shot0, int bs)
{
    if (!h->win) return (double)bs * h->g.Nz * h->g.Ny * h->g.Nx;
    double c = 0.0;
    for (int s = shot0; s < shot0 + bs; ++s) c += (double)h->g.Nz * (h->win_nx_h[s] + 2 * h->g.x0);
    return c;
}

// Copies each windowed shot's model into its slots (a no-op without windows).
lsrtm_status gather_model(lsrtm_handle *h, int shot0, int bs, bool born)
{
    if (!h->win) return LSRTM_OK;
    CU(launch_window_model(h->gm, h->g, h->win_x0_d, h->win_nx_d, shot0, bs, h->kdt, h->binv,
                           born ? h->kd2 : nullptr, born ? h->br2 : nullptr, h->st[0], h->st[1], h->sstride,
                           h->work));
    return LSRTM_OK;
}

// Runs `body` (kernel launches of one loop over a batch), captured once into a
// CUDA graph per (kind, batch) and replayed afterwards; nlaunch kernel
// launches and nsteps time steps of the batch are accounted to timing kind tkind.
template <class F>
lsrtm_status run_loop_n(lsrtm_handle *h, int kind, int tkind, int shot0, int bs, long long nlaunch,
                        long long nsteps, F &&body)
{
    const long long g0 = h->guard_count;
    long long guards = 0;   // guard checks (guard_step) of the loop
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (h->timing) {
        ea = take_event(h);
        eb = take_event(h);
        if (ea) CU(cudaEventRecord(ea, h->work));
    }
    if (!use_graphs(h)) {
        CHECK(body());
        guards = h->guard_count - g0;
    } else {
        auto key = std::make_pair(kind, shot0);
        auto it = h->graphs.find(key);
        cudaGraphExec_t exec;
        if (it == h->graphs.end()) {
            CU(cudaStreamBeginCapture(h->work, cudaStreamCaptureModeThreadLocal));
            lsrtm_status s = body();
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(h->work, &graph);
            if (s != LSRTM_OK) {
                if (graph) cudaGraphDestroy(graph);
                return s;
            }
            if (e != cudaSuccess) return fail(LSRTM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess)
                return fail(LSRTM_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
            h->graphs[key] = exec;
            h->graph_guards[key] = guards = h->guard_count - g0;
        } else {
            exec = it->second;
            guards = h->graph_guards[key];
        }
        CU(cudaGraphLaunch(exec, h->work));
    }
    nlaunch += guards;
    h->launches += nlaunch;
    if (h->timing && ea && eb) {
        CU(cudaEventRecord(eb, h->work));
        double cells = batch_cells(h, shot0, bs) * (double)nsteps;
        h->pending.push_back({tkind, ea, eb, nlaunch, cells});
    } else {
        if (ea) h->event_pool.push_back(ea);
        if (eb) h->event_pool.push_back(eb);
    }
    return LSRTM_OK;
}

int batch_size(const lsrtm_handle *h, int shot0) { return std::min(h->batch, h->nshot - shot0); }

lsrtm_status adj3f_step(lsrtm_handle *h, int i, int n, int s0, const Bands &bands);
lsrtm_status adj3f_start(lsrtm_handle *h, int fs0, int s0, int bs);

// Non-finite guard after the step of time n of a time loop of kind `kind`;
// i counts the pass's steps from its start (n forward, nt-1-n in reverse
// time, also across checkpoint segments). Every guard_K steps it checks the first
// `planes` planes of each of bs slots of the state just written (the
// pressure, with its Born or adjoint partner where the slot holds pairs).
// Once the guard word is set the time-step kernels return at once; the host
// reads the word when the call synchronises (check_kernel_error).
lsrtm_status guard_step(lsrtm_handle *h, int kind, int i, int n, const float *st, long long sstride, int planes,
                        int bs)
{
    if (h->guard_K <= 0 || (i + 1) % h->guard_K) return LSRTM_OK;
    CU(launch_guard_state(st, sstride, planes * h->g.plane, bs, h->kerr + 1, guard_code(kind, n), h->work));
    h->guard_count++;
    return LSRTM_OK;
}

// TMA row maps of the 2D migration reading state buffer j, or null.
const Maps2D *maps2_of(const lsrtm_handle *h, int j) { return h->tma2d ? &h->m2d[j] : nullptr; }

// Slot stride of state buffer j (3D: the fused kernels' ping and pong differ).
long long slot_stride(const lsrtm_handle *h, int j) { return j ? h->sstride1 : h->sstride; }

lsrtm_status zero_slots(lsrtm_handle *h, int bs)
{
    CU(cudaMemsetAsync(h->st[0], 0, (size_t)bs * h->sstride * sizeof(float), h->work));
    if (h->st[1]) CU(cudaMemsetAsync(h->st[1], 0, (size_t)bs * h->sstride1 * sizeof(float), h->work));
    if (h->psiv) CU(cudaMemsetAsync(h->psiv, 0, (size_t)bs * h->vstride * sizeof(float), h->work));
    if (h->bands.stage)
        CU(cudaMemsetAsync(h->bands.stage, 0, (size_t)bs * 2 * h->bands.nb * sizeof(float), h->work));
    return LSRTM_OK;
}

// Background forward pass over all shots: saves the boundary bands of p and
// the normal velocity every step and the final state (p^{nt-1}, v^{nt-1/2});
// optionally accumulates the pseudo-Hessian diagonal.
lsrtm_status bg_forward(lsrtm_handle *h, bool hess)
{
    const long long plane = h->g.plane;
    const int nt = h->g.nt;
    if (hess) CU(cudaMemsetAsync(h->hess_acc, 0, h->nint * sizeof(double), h->work));
    for (int s0 = 0; s0 < h->nshot; s0 += h->batch) {
        int bs = batch_size(h, s0);
        CHECK(zero_slots(h, bs));
        if (hess) CU(cudaMemsetAsync(h->hess, 0, (size_t)bs * plane * sizeof(float), h->work));
        if (is3d(h)) {
            // in place: p^{nt-1} is copied out between the two stages of the last step
            CHECK(run_loop(h, hess ? G_BG_HESS : G_BG, s0, bs, [&]() -> lsrtm_status {
                Step3D a = step3_args(h, s0);
                for (int n = 0; n < nt; ++n) {
                    a.n = n;
                    if (n + 1 < nt) {
                        CU(launch_fwd3d(a, bs, true, hess, 3, h->work));
                    } else {
                        CU(launch_fwd3d(a, bs, true, hess, 1, h->work));
                        for (int s = 0; s < bs; ++s)
                            CU(cudaMemcpyAsync(h->final_state + (size_t)(s0 + s) * 4 * plane,
                                               h->st[0] + s * h->sstride, plane * sizeof(float),
                                               cudaMemcpyDeviceToDevice, h->work));
                        CU(launch_fwd3d(a, bs, true, hess, 2, h->work));
                    }
                    if (h->bands.fmt != BAND_F32) CU(launch_band_pack(h->bands, bs, s0, n, h->work));
                    CHECK(guard_step(h, GK_BACKGROUND, n, n, h->st[0], h->sstride, 1, bs));
                }
                return LSRTM_OK;
            }));
            for (int s = 0; s < bs; ++s)
                CU(cudaMemcpyAsync(h->final_state + (size_t)(s0 + s) * 4 * plane + plane,
                                   h->st[0] + s * h->sstride + 1 * plane, 3 * plane * sizeof(float),
                                   cudaMemcpyDeviceToDevice, h->work));
        } else {
            CHECK(run_loop(h, hess ? G_BG_HESS : G_BG, s0, bs, [&]() -> lsrtm_status {
                CHECK(gather_model(h, s0, bs, false));
                Step2D a = step_args(h, s0);
                for (int n = 0; n < nt; ++n) {
                    a.n = n;
                    a.in = h->st[n & 1];
                    a.out = h->st[(n + 1) & 1];
                    CU(launch_fwd2d(a, bs, false, true, hess, h->work));
                    if (h->bands.fmt != BAND_F32) CU(launch_band_pack(h->bands, bs, s0, n, h->work));
                    CHECK(guard_step(h, GK_BACKGROUND, n, n, a.out, h->sstride, 1, bs));
                }
                return LSRTM_OK;
            }));
            // final state: p^{nt-1} is the input of the last step, v^{nt-1/2} its output
            const float *pin = h->st[(nt - 1) & 1];
            const float *vout = h->st[nt & 1];
            for (int s = 0; s < bs; ++s) {
                float *fs = h->final_state + (size_t)(s0 + s) * 3 * plane;
                CU(cudaMemcpyAsync(fs, pin + s * h->sstride, plane * sizeof(float), cudaMemcpyDeviceToDevice,
                                   h->work));
                CU(cudaMemcpyAsync(fs + plane, vout + s * h->sstride + 1 * plane, 2 * plane * sizeof(float),
                                   cudaMemcpyDeviceToDevice, h->work));
            }
        }
        if (hess) {
            CU(launch_hess_accumulate(h->gm, h->g, h->hess, bs, s0, h->win ? h->win_x0_d : nullptr, h->win_nx_d,
                                      h->hess_acc, h->work));
            h->launches++;
        }
    }
    if (hess) {
        CU(launch_hess_finalize(h->gm, h->hess_acc, h->hess_img, h->work));
        h->launches++;
        h->hess_ready = true;
    }
    h->bg_cached = true;
    return LSRTM_OK;
}

// Born modelling of the perturbation already prepared in h->kd2 / h->br2;
// records go to h->dstage.
lsrtm_status born_core(lsrtm_handle *h)
{
    const int nt = h->g.nt;
    for (int s0 = 0; s0 < h->nshot; s0 += h->batch) {
        int bs = batch_size(h, s0);
        CHECK(zero_slots(h, bs));
        CHECK(run_loop(h, G_BORN, s0, bs, [&]() -> lsrtm_status {
            if (is3d(h)) {
                for (int n = 0; n < nt; ++n) {
                    Step3F &a = h->f3born[n & 1];
                    a.n = n;
                    a.shot0 = s0;
                    a.trec = h->trv;
                    a.tzc = h->tzc;
                    CU(launch_born3f(a, bs, h->work));
                    CHECK(guard_step(h, GK_BORN, n, n, a.out, slot_stride(h, 1 - (n & 1)), 2, bs));
                }
                return LSRTM_OK;
            }
            CHECK(gather_model(h, s0, bs, true));
            Step2D a = step_args(h, s0);
            for (int n = 0; n < nt; ++n) {
                a.n = n;
                a.in = h->st[n & 1];
                a.out = h->st[(n + 1) & 1];
                CU(launch_fwd2d(a, bs, true, false, false, h->work, maps2_of(h, n & 1)));
                CHECK(guard_step(h, GK_BORN, n, n, a.out, h->sstride, 2, bs));
            }
            return LSRTM_OK;
        }));
    }
    return LSRTM_OK;
}

// Nonlinear modelling (Eq. 1) of every shot in the handle's own model: the
// background time loop with the pressure p^{n+1} recorded into h->dstage.
lsrtm_status model_core(lsrtm_handle *h)
{
    const int nt = h->g.nt;
    for (int s0 = 0; s0 < h->nshot; s0 += h->batch) {
        int bs = batch_size(h, s0);
        CHECK(zero_slots(h, bs));
        CHECK(run_loop(h, G_MODEL, s0, bs, [&]() -> lsrtm_status {
            if (is3d(h)) {
                Step3D a = step3_args(h, s0);
                a.rec_bg = 1;
                for (int n = 0; n < nt; ++n) {
                    a.n = n;
                    CU(launch_fwd3d(a, bs, false, false, 3, h->work));
                    CHECK(guard_step(h, GK_MODELLING, n, n, h->st[0], h->sstride, 1, bs));
                }
                return LSRTM_OK;
            }
            CHECK(gather_model(h, s0, bs, false));
            Step2D a = step_args(h, s0);
            a.rec_bg = 1;
            for (int n = 0; n < nt; ++n) {
                a.n = n;
                a.in = h->st[n & 1];
                a.out = h->st[(n + 1) & 1];
                CU(launch_fwd2d(a, bs, false, false, false, h->work));
                CHECK(guard_step(h, GK_MODELLING, n, n, a.out, h->sstride, 1, bs));
            }
            return LSRTM_OK;
        }));
    }
    return LSRTM_OK;
}

// ---------------------------------------------------------------------------
// Checkpointed reconstruction. The forward background pass of a batch saves
// the full background state every K steps; the reverse pass then walks the
// K-step segments from last to first: it restores the segment's checkpoint,
// recomputes the background forward over the segment while saving its
// boundary bands (the same kernel and inputs as the boundary mode, so the
// same bits), and runs the reverse steps that read those bands.
// ---------------------------------------------------------------------------

size_t ck_esize(const lsrtm_handle *h) { return h->ck_fmt == BAND_F32 ? sizeof(float) : 2; }

char *ck_slot_base(lsrtm_handle *h, int j)
{
    return static_cast<char *>(h->ck_mem) + (size_t)j * h->batch * h->ck_planes * h->g.plane * ck_esize(h);
}

// Copies `planes` contiguous planes of each of bs slots (slot stride sstride
// floats) into, or out of, planes [p0, p0 + planes) of checkpoint j: FP32
// as they are, 16-bit with one scale per slot and plane (k_ck_pack).
lsrtm_status ck_copy(lsrtm_handle *h, int j, float *slots, long long sstride, int planes, int p0, int bs,
                     bool save)
{
    if (h->ck_fmt != BAND_F32) {
        float *amax = h->ck_amax + (size_t)j * h->batch * h->ck_planes;
        if (save)
            CU(launch_ck_pack(slots, sstride, h->g.plane, planes, p0, bs, h->ck_planes, h->ck_fmt, ck_slot_base(h, j),
                              amax, h->work));
        else
            CU(launch_ck_unpack(slots, sstride, h->g.plane, planes, p0, bs, h->ck_planes, h->ck_fmt,
                                ck_slot_base(h, j), amax, h->work));
        return LSRTM_OK;
    }
    const size_t fb = (size_t)h->g.plane * sizeof(float);
    float *ck = reinterpret_cast<float *>(ck_slot_base(h, j)) + (size_t)p0 * h->g.plane;
    const size_t ckpitch = (size_t)h->ck_planes * fb, spitch = (size_t)sstride * sizeof(float);
    if (save)
        CU(cudaMemcpy2DAsync(ck, ckpitch, slots, spitch, planes * fb, bs, cudaMemcpyDeviceToDevice, h->work));
    else
        CU(cudaMemcpy2DAsync(slots, spitch, ck, ckpitch, planes * fb, bs, cudaMemcpyDeviceToDevice, h->work));
    return LSRTM_OK;
}

enum { G_CKF = 4, G_CKF_HESS = 5, G_SEG = 100 };

// Kernel launches of the 16-bit checkpoint saves of one forward pass
// (calls: ck_copy calls per snapshot; two kernels each).
long long ck16_launches(const lsrtm_handle *h, int calls)
{
    return h->ck_fmt != BAND_F32 ? 2LL * calls * h->ck_nseg : 0;
}

// Forward background pass of one batch in the main slots: checkpoints every K
// steps, the final state (p^{nt-1}, v^{nt-1/2}) of each shot of the batch into
// the batch-local final-state store, and optionally the pseudo-Hessian.
lsrtm_status ck_forward(lsrtm_handle *h, int s0, int bs, bool hess)
{
    const long long plane = h->g.plane;
    const int nt = h->g.nt, K = h->ck_K;
    CHECK(zero_slots(h, bs));
    if (hess) CU(cudaMemsetAsync(h->hess, 0, (size_t)bs * plane * sizeof(float), h->work));
    if (is3d(h)) {
        CHECK(run_loop_n(h, hess ? G_CKF_HESS : G_CKF, 1, s0, bs, 2LL * nt + ck16_launches(h, 1), nt, [&]() -> lsrtm_status {
            Step3D a = step3_args(h, s0);
            for (int n = 0; n < nt; ++n) {
                a.n = n;
                if (n % K == 0) CHECK(ck_copy(h, n / K, h->st[0], h->sstride, 10, 0, bs, true));
                if (n + 1 < nt) {
                    CU(launch_fwd3d(a, bs, false, hess, 3, h->work));
                    CHECK(guard_step(h, GK_BACKGROUND, n, n, h->st[0], h->sstride, 1, bs));
                    continue;
                }
                CU(launch_fwd3d(a, bs, false, hess, 1, h->work));
                CU(cudaMemcpy2DAsync(h->final_state, 4 * plane * sizeof(float), h->st[0], h->sstride * sizeof(float),
                                     plane * sizeof(float), bs, cudaMemcpyDeviceToDevice, h->work));
                CU(launch_fwd3d(a, bs, false, hess, 2, h->work));
            }
            return LSRTM_OK;
        }));
        CU(cudaMemcpy2DAsync(h->final_state + plane, 4 * plane * sizeof(float), h->st[0] + plane,
                             h->sstride * sizeof(float), 3 * plane * sizeof(float), bs, cudaMemcpyDeviceToDevice,
                             h->work));
    } else {
        CHECK(run_loop_n(h, hess ? G_CKF_HESS : G_CKF, 1, s0, bs, nt + ck16_launches(h, 2), nt, [&]() -> lsrtm_status {
            Step2D a = step_args(h, s0);
            for (int n = 0; n < nt; ++n) {
                a.n = n;
                a.in = h->st[n & 1];
                a.out = h->st[(n + 1) & 1];
                if (n % K == 0) {
                    CHECK(ck_copy(h, n / K, h->st[n & 1], h->sstride, 5, 0, bs, true));
                    CHECK(ck_copy(h, n / K, h->psiv, h->vstride, 2, 5, bs, true));
                }
                CU(launch_fwd2d(a, bs, false, false, hess, h->work));
                CHECK(guard_step(h, GK_BACKGROUND, n, n, a.out, h->sstride, 1, bs));
            }
            return LSRTM_OK;
        }));
        CU(cudaMemcpy2DAsync(h->final_state, 3 * plane * sizeof(float), h->st[(nt - 1) & 1],
                             h->sstride * sizeof(float), plane * sizeof(float), bs, cudaMemcpyDeviceToDevice,
                             h->work));
        CU(cudaMemcpy2DAsync(h->final_state + plane, 3 * plane * sizeof(float), h->st[nt & 1] + plane,
                             h->sstride * sizeof(float), 2 * plane * sizeof(float), bs, cudaMemcpyDeviceToDevice,
                             h->work));
    }
    if (hess) {
        CU(launch_hess_accumulate(h->gm, h->g, h->hess, bs, s0, nullptr, nullptr, h->hess_acc, h->work));
        h->launches++;
    }
    return LSRTM_OK;
}

// Reverse steps of segment j: n from min((j+1)K, nt-1) down to jK+1 (down to
// 0 for the first segment); they read the bands of steps jK .. hi-1.
void seg_range(const lsrtm_handle *h, int j, int *t0, int *hi, int *lo)
{
    *t0 = j * h->ck_K;
    *hi = std::min((j + 1) * h->ck_K, h->g.nt - 1);
    *lo = j == 0 ? 0 : *t0 + 1;
}

// Restores checkpoint j and recomputes the background over steps t0 .. hi-1
// into the segment band buffer.
lsrtm_status ck_recompute(lsrtm_handle *h, int s0, int bs, int j)
{
    int t0, hi, lo;
    seg_range(h, j, &t0, &hi, &lo);
    const long long plane = h->g.plane;
    const long long c = hi - t0;
    Bands sb = h->segbands;
    sb.shot0 = s0;
    sb.t0 = t0;
    const bool d3 = is3d(h);
    const bool pack = sb.fmt != BAND_F32;
    const long long unpack = h->ck_fmt != BAND_F32 ? (d3 ? 1 : 2) : 0;   // 16-bit checkpoint restores
    return run_loop_n(h, G_SEG + 2 * j, 1, s0, bs, (d3 ? 2 * c : c) + (pack ? c : 0) + unpack, c,
                      [&]() -> lsrtm_status {
        if (d3) {
            CHECK(ck_copy(h, j, h->rec[0], 10 * plane, 10, 0, bs, false));
            Step3D a = step3_args(h, s0);
            a.st = h->rec[0];
            a.sstride = 10 * plane;
            a.bands = sb;
            for (int n = t0; n < hi; ++n) {
                a.n = n;
                CU(launch_fwd3d(a, bs, true, false, 3, h->work));
                if (pack) CU(launch_band_pack(sb, bs, s0, n, h->work));
                CHECK(guard_step(h, GK_RECOMPUTE, n, n, a.st, a.sstride, 1, bs));
            }
            return LSRTM_OK;
        }
        CHECK(ck_copy(h, j, h->rec[t0 & 1], 5 * plane, 5, 0, bs, false));
        CHECK(ck_copy(h, j, h->rec_psiv, 2 * plane, 2, 5, bs, false));
        Step2D a = step_args(h, s0);
        a.sstride = 5 * plane;
        a.vstride = 2 * plane;
        a.psiv = h->rec_psiv;
        a.bands = sb;
        for (int n = t0; n < hi; ++n) {
            a.n = n;
            a.in = h->rec[n & 1];
            a.out = h->rec[(n + 1) & 1];
            CU(launch_fwd2d(a, bs, false, true, false, h->work));
            if (pack) CU(launch_band_pack(sb, bs, s0, n, h->work));
            CHECK(guard_step(h, GK_RECOMPUTE, n, n, a.out, a.sstride, 1, bs));
        }
        return LSRTM_OK;
    });
}

// The reverse (adjoint) steps of segment j.
lsrtm_status ck_reverse(lsrtm_handle *h, int s0, int bs, int j)
{
    int t0, hi, lo;
    seg_range(h, j, &t0, &hi, &lo);
    const int nt = h->g.nt;
    const long long r = hi - lo + 1;
    Bands sb = h->segbands;
    sb.shot0 = s0;
    sb.t0 = t0;
    const bool d3 = is3d(h);
    return run_loop_n(h, G_SEG + 2 * j + 1, 2, s0, bs, r, r, [&]() -> lsrtm_status {
        if (d3) {
            for (int n = hi; n >= lo; --n) {
                CHECK(adj3f_step(h, nt - 1 - n, n, s0, sb));
                const int o = 1 - ((nt - 1 - n) & 1);
                CHECK(guard_step(h, GK_MIGRATION, nt - 1 - n, n, h->st[o], slot_stride(h, o), 2, bs));
            }
            return LSRTM_OK;
        }
        Step2D a = step_args(h, s0);
        a.bands = sb;
        for (int n = hi; n >= lo; --n) {
            const int i = nt - 1 - n;
            a.n = n;
            a.in = h->st[i & 1];
            a.out = h->st[(i + 1) & 1];
            CU(launch_adj2d(a, maps2_of(h, i & 1), bs, h->work));
            CHECK(guard_step(h, GK_MIGRATION, nt - 1 - n, n, a.out, h->sstride, 2, bs));
        }
        return LSRTM_OK;
    });
}

// Pseudo-Hessian only (checkpoint mode has no cached background pass).
lsrtm_status ck_hessian(lsrtm_handle *h)
{
    CU(cudaMemsetAsync(h->hess_acc, 0, h->nint * sizeof(double), h->work));
    for (int s0 = 0; s0 < h->nshot; s0 += h->batch) CHECK(ck_forward(h, s0, batch_size(h, s0), true));
    CU(launch_hess_finalize(h->gm, h->hess_acc, h->hess_img, h->work));
    h->launches++;
    h->hess_ready = true;
    return LSRTM_OK;
}

lsrtm_status adjoint_core_ckpt(lsrtm_handle *h, float *gout, bool want_hess)
{
    const long long plane = h->g.plane;
    const int nt = h->g.nt;
    const bool hess = want_hess && !h->hess_ready;
    if (hess) CU(cudaMemsetAsync(h->hess_acc, 0, h->nint * sizeof(double), h->work));
    CU(cudaMemsetAsync(h->img_acc, 0, h->nint * sizeof(double2), h->work));
    for (int s0 = 0; s0 < h->nshot; s0 += h->batch) {
        int bs = batch_size(h, s0);
        CHECK(ck_forward(h, s0, bs, hess));
        CHECK(zero_slots(h, bs));
        if (h->img) CU(cudaMemsetAsync(h->img, 0, (size_t)bs * plane * sizeof(float2), h->work));
        if (is3d(h)) {
            CHECK(adj3f_start(h, 0, s0, bs));
        } else {
            CU(launch_pack_adjoint(h->g, h->final_state, 0, bs, h->st[0], h->sstride, h->work));
            CU(launch_inject_residual(h->g, h->trv, bs, s0, h->dstage, nt - 1,
                                      reinterpret_cast<float2 *>(h->st[0]), h->sstride / 2, h->work));
            h->launches += 2;
        }
        for (int j = h->ck_nseg - 1; j >= 0; --j) {
            int t0, hi, lo;
            seg_range(h, j, &t0, &hi, &lo);
            if (hi < lo) continue;
            CHECK(ck_recompute(h, s0, bs, j));
            CHECK(ck_reverse(h, s0, bs, j));
        }
        CU(launch_image_accumulate(h->gm, h->g, h->img, bs, s0, nullptr, nullptr, h->img_acc, h->work));
        h->launches++;
    }
    if (hess) {
        CU(launch_hess_finalize(h->gm, h->hess_acc, h->hess_img, h->work));
        h->launches++;
        h->hess_ready = true;
    }
    CU(launch_image_finalize(h->gm, h->img_acc, h->kdt, h->binv, gout, h->work));
    h->launches++;
    return LSRTM_OK;
}

// L^T of the data in h->dstage; stacked images into h->img_acc, then the
// chain rule into gout ([2][nint], device).
lsrtm_status adjoint_core(lsrtm_handle *h, float *gout, bool want_hess)
{
    if (h->ckpt) return adjoint_core_ckpt(h, gout, want_hess);
    const long long plane = h->g.plane;
    const int nt = h->g.nt;
    if (!h->bg_cached || h->cfg.plan == LSRTM_PLAN_PLAIN || (want_hess && !h->hess_ready))
        CHECK(bg_forward(h, want_hess && !h->hess_ready));
    CU(cudaMemsetAsync(h->img_acc, 0, h->nint * sizeof(double2), h->work));
    for (int s0 = 0; s0 < h->nshot; s0 += h->batch) {
        int bs = batch_size(h, s0);
        CHECK(zero_slots(h, bs));
        if (h->img) CU(cudaMemsetAsync(h->img, 0, (size_t)bs * plane * sizeof(float2), h->work));
        if (is3d(h)) {
            CHECK(adj3f_start(h, s0, s0, bs));
            CHECK(run_loop(h, G_ADJ, s0, bs, [&]() -> lsrtm_status {
                for (int i = 0; i < nt; ++i) {
                    CHECK(adj3f_step(h, i, nt - 1 - i, s0, h->bands));
                    const int o = 1 - (i & 1);
                    CHECK(guard_step(h, GK_MIGRATION, i, nt - 1 - i, h->st[o], slot_stride(h, o), 2, bs));
                }
                return LSRTM_OK;
            }));
            CU(launch_image_accumulate(h->gm, h->g, h->img, bs, s0, nullptr, nullptr, h->img_acc, h->work));
            h->launches++;
        } else {
            CU(launch_pack_adjoint(h->g, h->final_state, s0, bs, h->st[0], h->sstride, h->work));
            CU(launch_inject_residual(h->g, h->trv, bs, s0, h->dstage, nt - 1,
                                      reinterpret_cast<float2 *>(h->st[0]), h->sstride / 2, h->work));
            h->launches += 2;
            CHECK(run_loop(h, G_ADJ, s0, bs, [&]() -> lsrtm_status {
                CHECK(gather_model(h, s0, bs, false));
                Step2D a = step_args(h, s0);
                for (int i = 0; i < nt; ++i) {
                    a.n = nt - 1 - i;
                    a.in = h->st[i & 1];
                    a.out = h->st[(i + 1) & 1];
                    CU(launch_adj2d(a, maps2_of(h, i & 1), bs, h->work));
                    CHECK(guard_step(h, GK_MIGRATION, i, nt - 1 - i, a.out, h->sstride, 2, bs));
                }
                return LSRTM_OK;
            }));
            CU(launch_image_accumulate(h->gm, h->g, h->img, bs, s0, h->win ? h->win_x0_d : nullptr, h->win_nx_d,
                                       h->img_acc, h->work));
            h->launches++;
        }
    }
    CU(launch_image_finalize(h->gm, h->img_acc, h->kdt, h->binv, gout, h->work));
    h->launches++;
    return LSRTM_OK;
}

lsrtm_status prep_perturbation(lsrtm_handle *h, const float *dm_dev)
{
    CU(launch_pert_prep(h->gm, dm_dev, h->kdt, h->binv, h->kd2, h->br2, h->work));
    h->launches++;
    return LSRTM_OK;
}

lsrtm_status check_finite(lsrtm_handle *h, const float *x, long long n, const char *what)
{
    CU(cudaMemsetAsync(h->flag, 0, sizeof(int), h->work));
    CU(launch_nonfinite_count(x, n, h->flag, h->work));
    h->launches++;
    int flag = 0;
    CU(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->work));
    CU(cudaStreamSynchronize(h->work));
    if (flag) return fail(LSRTM_ERR_NONFINITE, std::string("non-finite values in ") + what);
    return LSRTM_OK;
}

lsrtm_status validate_cfg(const lsrtm_config *c)
{
    if (!c) return fail(LSRTM_ERR_ARG, "null config");
    if (c->ndim != 2 && c->ndim != 3) return fail(LSRTM_ERR_ARG, "ndim must be 2 or 3");
    if (c->ndim == 3 && (c->ny < 1 || !(c->dy > 0))) return fail(LSRTM_ERR_ARG, "3D needs ny >= 1 and dy > 0");
    if (c->fd_order != 4 && c->fd_order != 8) return fail(LSRTM_ERR_ARG, "fd_order must be 4 or 8");
    if (c->nz < 1 || c->nx < 1 || c->nt < 1) return fail(LSRTM_ERR_ARG, "empty grid or nt < 1");
    if (c->npml < c->fd_order / 2) return fail(LSRTM_ERR_ARG, "npml must be >= fd_order/2");
    if (!(c->dt > 0) || !(c->dx > 0) || !(c->dz > 0)) return fail(LSRTM_ERR_ARG, "non-positive spacing or dt");
    if (c->band_precision != LSRTM_BAND_FP32 && c->band_precision != LSRTM_BAND_BF16 &&
        c->band_precision != LSRTM_BAND_FP16)
        return fail(LSRTM_ERR_ARG, "band_precision must be 0 (fp32), 1 (bf16) or 2 (fp16)");
    if (c->checkpoint_precision != LSRTM_BAND_FP32 && c->checkpoint_precision != LSRTM_BAND_BF16 &&
        c->checkpoint_precision != LSRTM_BAND_FP16)
        return fail(LSRTM_ERR_ARG, "checkpoint_precision must be 0 (fp32), 1 (bf16) or 2 (fp16)");
    if (c->recon_mode != LSRTM_RECON_BOUNDARY && c->recon_mode != LSRTM_RECON_CHECKPOINT &&
        c->recon_mode != LSRTM_RECON_AUTO)
        return fail(LSRTM_ERR_ARG, "recon_mode must be 0 (boundary), 1 (checkpoint) or 2 (auto)");
    if (c->plan != LSRTM_PLAN_BATCHED && c->plan != LSRTM_PLAN_PLAIN)
        return fail(LSRTM_ERR_ARG, "unknown plan");
    if (c->shots_per_batch < 0) return fail(LSRTM_ERR_ARG, "shots_per_batch < 0");
    if (c->checkpoint_interval < 0) return fail(LSRTM_ERR_ARG, "checkpoint_interval < 0");
    if (c->free_surface != 0 && c->free_surface != 1) return fail(LSRTM_ERR_ARG, "free_surface must be 0 or 1");
    if (c->free_surface && c->nz < c->fd_order)
        return fail(LSRTM_ERR_ARG, "a free surface needs nz >= fd_order (its mirror rows)");
    return LSRTM_OK;
}

// Receivers of every 2D shot grouped by the CTA tile (txo columns x tzc rows)
// that records them: CSR over shot * ntiles + tile, cells sorted within a tile.
lsrtm_status build_tiles(lsrtm_handle *h)
{
    const GridDev &g = h->g;
    // 2D: CTA tiles of txo columns x tzc rows; 3D: kTile3X x kTile3Y columns x tzc rows
    const bool d3 = g.ndim == 3;
    const int tw = d3 ? kTile3X : h->txo;
    int ntx = (g.Nx + tw - 1) / tw, ntz = (g.Nz + h->tzc - 1) / h->tzc;
    int nty = d3 ? (g.Ny + kTile3Y - 1) / kTile3Y : 1;
    int ntiles = ntx * nty * ntz;
    std::vector<std::vector<int2>> lists((size_t)h->nshot * ntiles);
    for (int s = 0; s < h->nshot; ++s)
        for (int r = h->rec_ptr[s]; r < h->rec_ptr[s + 1]; ++r) {
            int2 e = h->rec_cells_h[r];
            int z = (int)(e.x / g.rowz), y = (int)((e.x % g.rowz) / g.pitch), x = (int)(e.x % g.pitch);
            int t = ((z / h->tzc) * nty + (d3 ? y / kTile3Y : 0)) * ntx + x / tw;
            lists[(size_t)s * ntiles + t].push_back(e);
        }
    std::vector<int> ptr(lists.size() + 1, 0);
    std::vector<int2> flat;
    flat.reserve(h->nrec_total);
    for (size_t i = 0; i < lists.size(); ++i) {
        auto &L = lists[i];
        std::stable_sort(L.begin(), L.end(), [](int2 a, int2 b) { return a.x < b.x; });
        flat.insert(flat.end(), L.begin(), L.end());
        ptr[i + 1] = (int)flat.size();
    }
    if (ptr.size() > h->trec_ptr_cap) {
        CHECK(dalloc_t(h, &h->trec_ptr, ptr.size()));
        h->trec_ptr_cap = ptr.size();
    }
    CU(cudaMemcpyAsync(h->trec_ptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice, h->work));
    if (!flat.empty())
        CU(cudaMemcpyAsync(h->trec, flat.data(), flat.size() * sizeof(int2), cudaMemcpyHostToDevice, h->work));
    CU(cudaStreamSynchronize(h->work));
    h->trv.ptr = h->trec_ptr;
    h->trv.rec = h->trec;
    h->trv.ntiles = ntiles;
    return LSRTM_OK;
}

lsrtm_status build_geometry(lsrtm_handle *h, const lsrtm_geometry *geo)
{
    const GridDev &g = h->g;
    if (!geo || geo->nshot < 1 || !geo->src_idx || !geo->rec_ptr || (!geo->rec_idx && geo->rec_ptr[geo->nshot] > 0))
        return fail(LSRTM_ERR_ARG, "invalid geometry");
    h->nshot = geo->nshot;
    if (geo->rec_ptr[0] != 0) return fail(LSRTM_ERR_GEOMETRY, "rec_ptr[0] must be 0");
    for (int s = 0; s < h->nshot; ++s)
        if (geo->rec_ptr[s + 1] < geo->rec_ptr[s]) return fail(LSRTM_ERR_GEOMETRY, "rec_ptr not monotone");
    h->nrec_total = geo->rec_ptr[h->nshot];
    h->rec_ptr.assign(geo->rec_ptr, geo->rec_ptr + h->nshot + 1);
    const GridDev &gm = h->gm;
    h->rec_off_h.assign(h->nrec_total, 0.0);
    for (int s = 0; s < h->nshot; ++s) {
        const long long ks = geo->src_idx[s];
        const long long xs = ks % gm.nx, ys = (ks / gm.nx) % gm.ny;
        for (int r = geo->rec_ptr[s]; r < geo->rec_ptr[s + 1]; ++r) {
            const long long k = geo->rec_idx[r];
            const long long xr = k % gm.nx, yr = (k / gm.nx) % gm.ny;
            h->rec_off_h[r] = std::hypot((double)(xr - xs) * h->cfg.dx, (double)(yr - ys) * h->cfg.dy);
        }
    }
    // cell of interior point k in shot s's slot grid (its window), or -1 outside the window
    auto pad_cell = [&](long long k, int s) -> long long {
        long long ix = k % gm.nx, t = k / gm.nx, iy = t % gm.ny, iz = t / gm.ny;
        if (h->win) {
            ix -= h->win_x0_h[s];
            if (ix < 0 || ix >= h->win_nx_h[s]) return -1;
        }
        return (iz + g.z0) * g.rowz + (iy + g.y0) * g.pitch + (ix + g.x0);
    };
    std::vector<int> src(h->nshot);
    for (int s = 0; s < h->nshot; ++s) {
        long long k = geo->src_idx[s];
        if (k < 0 || k >= h->nint) return fail(LSRTM_ERR_GEOMETRY, "source outside the interior grid");
        long long c = pad_cell(k, s);
        if (c < 0) return fail(LSRTM_ERR_GEOMETRY, "source outside its shot's aperture window");
        if (g.fs && k / ((long long)gm.nx * gm.ny) == 0)
            return fail(LSRTM_ERR_GEOMETRY, "a source on the free-surface row radiates nothing (p = 0 there)");
        src[s] = (int)c;
    }
    if (g.ndim == 3) {
        // per shot: receivers sorted by cell, and a node map to the first receiver at each node
        std::vector<int> rptr(h->nshot + 1, 0), rcell, rrow;
        rcell.reserve(h->nrec_total);
        rrow.reserve(h->nrec_total);
        for (int s = 0; s < h->nshot; ++s) {
            std::vector<std::pair<long long, int>> L;
            for (int r = geo->rec_ptr[s]; r < geo->rec_ptr[s + 1]; ++r) {
                long long k = geo->rec_idx[r];
                if (k < 0 || k >= h->nint) return fail(LSRTM_ERR_GEOMETRY, "receiver outside the interior grid");
                L.emplace_back(pad_cell(k, s), r);
            }
            std::stable_sort(L.begin(), L.end(),
                             [](const std::pair<long long, int> &a, const std::pair<long long, int> &b) {
                                 return a.first < b.first;
                             });
            for (auto &e : L) {
                rcell.push_back((int)e.first);
                rrow.push_back(e.second);
            }
            rptr[s + 1] = (int)rcell.size();
        }
        CHECK(dalloc_t(h, &h->src_cell, src.size()));
        CHECK(dalloc_t(h, &h->rptr, rptr.size()));
        CHECK(dalloc_t(h, &h->rcell, std::max<size_t>(rcell.size(), 1)));
        CHECK(dalloc_t(h, &h->rrow, std::max<size_t>(rrow.size(), 1)));
        CHECK(dalloc_t(h, &h->rmap, (size_t)h->nshot * g.plane));
        CU(cudaMemsetAsync(h->rmap, 0xff, (size_t)h->nshot * g.plane * sizeof(int), h->work));   // -1
        CU(cudaMemcpyAsync(h->src_cell, src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice, h->work));
        CU(cudaMemcpyAsync(h->rptr, rptr.data(), rptr.size() * sizeof(int), cudaMemcpyHostToDevice, h->work));
        if (!rcell.empty()) {
            CU(cudaMemcpyAsync(h->rcell, rcell.data(), rcell.size() * sizeof(int), cudaMemcpyHostToDevice, h->work));
            CU(cudaMemcpyAsync(h->rrow, rrow.data(), rrow.size() * sizeof(int), cudaMemcpyHostToDevice, h->work));
        }
        // first receiver of each node of each shot
        for (int s = 0; s < h->nshot; ++s)
            CU(launch_rmap_scatter(h->rmap + (size_t)s * g.plane, h->rcell, rptr[s], rptr[s + 1], h->work));
        CU(cudaStreamSynchronize(h->work));
        // receivers per fused-kernel tile
        h->rec_cells_h.resize(h->nrec_total);
        for (int s = 0; s < h->nshot; ++s)
            for (int r = geo->rec_ptr[s]; r < geo->rec_ptr[s + 1]; ++r)
                h->rec_cells_h[r] = make_int2((int)pad_cell(geo->rec_idx[r], s), r);
        CHECK(dalloc_t(h, &h->trec, std::max<size_t>(h->rec_cells_h.size(), 1)));
        return build_tiles(h);
    }
    h->rec_cells_h.resize(h->nrec_total);
    for (int s = 0; s < h->nshot; ++s)
        for (int r = geo->rec_ptr[s]; r < geo->rec_ptr[s + 1]; ++r) {
            long long k = geo->rec_idx[r];
            if (k < 0 || k >= h->nint) return fail(LSRTM_ERR_GEOMETRY, "receiver outside the interior grid");
            long long cell = pad_cell(k, s);
            if (cell < 0) return fail(LSRTM_ERR_GEOMETRY, "receiver outside its shot's aperture window");
            h->rec_cells_h[r] = make_int2((int)cell, r);
        }
    CHECK(dalloc_t(h, &h->src_cell, src.size()));
    CU(cudaMemcpyAsync(h->src_cell, src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice, h->work));
    CHECK(dalloc_t(h, &h->trec, std::max<size_t>(h->rec_cells_h.size(), 1)));
    return build_tiles(h);
}

// Aperture windows: validates them, keeps host and device copies and turns
// h->g into the slot grid of the widest window (h->gm stays the model grid).
lsrtm_status setup_windows(lsrtm_handle *h, const lsrtm_geometry *geo)
{
    if (!geo || (!geo->win_x0 && !geo->win_nx)) return LSRTM_OK;
    if (!geo->win_x0 || !geo->win_nx) return fail(LSRTM_ERR_ARG, "win_x0 and win_nx must both be given or both NULL");
    if (h->g.ndim != 2) return fail(LSRTM_ERR_ARG, "aperture windows are supported in 2D only");
    if (geo->nshot < 1) return fail(LSRTM_ERR_ARG, "invalid geometry");
    h->win_x0_h.assign(geo->win_x0, geo->win_x0 + geo->nshot);
    h->win_nx_h.assign(geo->win_nx, geo->win_nx + geo->nshot);
    int wmax = 0;
    for (int s = 0; s < geo->nshot; ++s) {
        int x0 = h->win_x0_h[s], nx = h->win_nx_h[s];
        if (x0 < 0 || nx < 1 || (long long)x0 + nx > h->gm.nx)
            return fail(LSRTM_ERR_GEOMETRY, "aperture window outside the model");
        wmax = std::max(wmax, nx);
    }
    h->win = true;
    GridDev &g = h->g;
    g.nx = wmax;
    g.Nx = wmax + 2 * g.x0;
    g.pitch = (g.Nx + 31) / 32 * 32;
    g.rowz = (long long)g.Ny * g.pitch;
    g.plane = (long long)g.Nz * g.rowz;
    CHECK(dalloc_t(h, &h->win_x0_d, geo->nshot));
    CHECK(dalloc_t(h, &h->win_nx_d, geo->nshot));
    CU(cudaMemcpyAsync(h->win_x0_d, h->win_x0_h.data(), geo->nshot * sizeof(int), cudaMemcpyHostToDevice, h->work));
    CU(cudaMemcpyAsync(h->win_nx_d, h->win_nx_h.data(), geo->nshot * sizeof(int), cudaMemcpyHostToDevice, h->work));
    CU(cudaStreamSynchronize(h->work));
    return LSRTM_OK;
}

// Arguments of the fused 3D Born step reading buffer `b` (0: st[0], 1: st[1]),
// with its tensor maps; the launches change only n, in/out and shot0.
lsrtm_status setup_fused3d(lsrtm_handle *h)
{
    // the kernels index within a slot with 32-bit offsets
    if (std::max(h->sstride, h->sstride1) >= (1LL << 31))
        return fail(LSRTM_ERR_ARG, "3D grid too large for the fused kernels (slot above 2^31 floats)");
    for (int b = 0; b < 2; ++b) {
        Step3F &a = h->f3born[b];
        a = Step3F{};
        a.g = h->g;
        a.pml = h->pml;
        a.in = h->st[b];
        a.out = h->st[1 - b];
        a.in_pairs = (int)((b ? h->sstride1 : h->sstride) / (2 * h->g.plane));
        a.out_pairs = (int)((b ? h->sstride : h->sstride1) / (2 * h->g.plane));
        a.psiv = h->st[0] + 2LL * kBornPairs3F * h->g.plane;
        a.psiv_pairs = (int)(h->sstride / (2 * h->g.plane));
        a.br2 = h->br2;
        a.tzc = h->tzc;
        a.wav = h->wav;
        a.wav_per_shot = h->cfg.wavelet_per_shot;
        a.src_cell = h->src_cell;
        a.src_scale = h->src_scale;
        a.dstage = h->dstage;
        a.err = h->kerr;
        cudaError_t e = fused3d_born_maps(a, h->kd2, h->br2, h->batch);
        if (e != cudaSuccess) return fail(LSRTM_ERR_CUDA, std::string("tensor maps: ") + cudaGetErrorString(e));
        Adj3F &d = h->f3adj[b];
        d = Adj3F{};
        d.g = h->g;
        d.pml = h->pml;
        d.in = h->st[b];
        d.out = h->st[1 - b];
        d.in_planes = (int)((b ? h->sstride1 : h->sstride) / h->g.plane);
        d.out_planes = (int)((b ? h->sstride : h->sstride1) / h->g.plane);
        d.kdt = h->kdt;
        d.binv = h->binv;
        d.img = h->img;
        d.tzc = h->tzc;
        d.wav = h->wav;
        d.wav_per_shot = h->cfg.wavelet_per_shot;
        d.src_cell = h->src_cell;
        d.src_scale = h->src_scale;
        d.dstage = h->dstage;
        d.err = h->kerr;
        e = fused3d_adj_maps(d, h->kdt, h->binv, h->batch);
        if (e != cudaSuccess) return fail(LSRTM_ERR_CUDA, std::string("tensor maps: ") + cudaGetErrorString(e));
    }
    return LSRTM_OK;
}

// One fused 3D adjoint step n of a batch; i = nt - 1 - n selects the input buffer.
lsrtm_status adj3f_step(lsrtm_handle *h, int i, int n, int s0, const Bands &bands)
{
    Adj3F &a = h->f3adj[i & 1];
    a.n = n;
    a.shot0 = s0;
    a.bands = bands;
    a.trec = h->trv;
    a.tzc = h->tzc;
    CU(launch_adj3f(a, batch_size(h, s0), h->work));
    return LSRTM_OK;
}

// Start of a fused 3D reverse pass: (p, 0), (v, 0) from the saved final
// states (fs0: index of the batch's first shot in the final-state store) and
// the residual of step nt-1 added to lambda_p.
lsrtm_status adj3f_start(lsrtm_handle *h, int fs0, int s0, int bs)
{
    CU(launch_pack3f(h->g, h->final_state, fs0, bs, h->st[0], h->sstride, h->work));
    CU(launch_inject_residual(h->g, h->trv, bs, s0, h->dstage, h->g.nt - 1, reinterpret_cast<float2 *>(h->st[0]),
                              h->sstride / 2, h->work));
    h->launches += 2;
    return LSRTM_OK;
}

// Reads and clears the device error words (synchronises the work stream):
// the fused kernels' tile-copy word and the non-finite guard word.
lsrtm_status check_kernel_error(lsrtm_handle *h)
{
    if (!h->kerr) return LSRTM_OK;
    int e[2] = {0, 0};
    CU(cudaMemcpyAsync(e, h->kerr, sizeof(e), cudaMemcpyDeviceToHost, h->work));
    CU(cudaStreamSynchronize(h->work));
    if (!e[0] && !e[1]) return LSRTM_OK;
    CU(cudaMemsetAsync(h->kerr, 0, sizeof(e), h->work));
    CU(cudaStreamSynchronize(h->work));
    if (e[0])
        return fail(LSRTM_ERR_CUDA, (e[0] & 2) ? "a fused 3D kernel refused a misaligned tile copy"
                                               : "a fused 3D kernel gave up waiting for its tile copies");
    const int kind = e[1] >> 24, n = (e[1] & 0xFFFFFF) - 1;
    if (kind == GK_CG)
        return fail(LSRTM_ERR_NONFINITE, "non-finite CG scalar (<q,q>, gamma or <r,r>) at iteration " +
                                             std::to_string(n));
    static const char *names[] = {"?", "background", "Born", "migration", "nonlinear modelling",
                                  "checkpoint recomputation"};
    return fail(LSRTM_ERR_NONFINITE, std::string("non-finite wavefield in the ") +
                                         names[kind >= 1 && kind <= 5 ? kind : 0] + " time loop at step " +
                                         std::to_string(n) + "; the rest of the loop was skipped");
}

int geo_nshot(const lsrtm_geometry *geo) { return geo && geo->nshot > 0 ? geo->nshot : 1; }

lsrtm_status create_impl(const lsrtm_config *cfg, const float *vp, const float *rho,
                         const float *wavelet, const lsrtm_geometry *geo, void *stream,
                         lsrtm_handle *h)
{
    CHECK(validate_cfg(cfg));
    h->cfg = *cfg;
    h->user = (cudaStream_t)stream;
    CU(cudaStreamCreateWithFlags(&h->work, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    CU(cudaEventRecord(h->ev_in, h->user));
    CU(cudaStreamWaitEvent(h->work, h->ev_in, 0));
    CU(ensure_kernels_configured());

    GridDev &g = h->g;
    g.ndim = cfg->ndim;
    g.M = cfg->fd_order / 2;
    const bool d3 = cfg->ndim == 3;
    g.nz = cfg->nz;
    g.ny = d3 ? cfg->ny : 1;
    g.nx = cfg->nx;
    g.z0 = cfg->npml;
    g.y0 = d3 ? cfg->npml : 0;
    g.x0 = cfg->npml;
    g.Nz = g.nz + 2 * cfg->npml;
    g.Ny = d3 ? g.ny + 2 * cfg->npml : 1;
    g.Nx = g.nx + 2 * cfg->npml;
    g.pitch = (g.Nx + 31) / 32 * 32;
    g.rowz = (long long)g.Ny * g.pitch;
    g.plane = (long long)g.Nz * g.rowz;
    g.dt = (float)cfg->dt;
    g.nt = cfg->nt;
    g.fs = cfg->free_surface ? 1 : 0;
    double c[4];
    fd_coeffs(g.M, c);
    for (int l = 0; l < kMaxM; ++l) {
        double cl = l < g.M ? c[l] : 0.0;
        g.cz[l] = (float)(cl / cfg->dz);
        g.cy[l] = (float)(cl / (cfg->dy > 0 ? cfg->dy : 1.0));
        g.cx[l] = (float)(cl / cfg->dx);
    }
    h->nint = (long long)g.nz * g.ny * g.nx;
    // CTA blocking: output columns fixed by the kernel, z-chunks of about 112 rows
    h->txo = march2d_txo(g.M);
    if (d3) {
        // enough CTAs for two waves of one CTA per SM, chunks of at least 8M rows
        const int ntxy = ((g.Nx + kTile3X - 1) / kTile3X) * ((g.Ny + kTile3Y - 1) / kTile3Y);
        const int want = (2 * 152 + ntxy * geo_nshot(geo) - 1) / std::max(1, ntxy * geo_nshot(geo));
        const int nchunk = std::max(1, std::min(want, g.Nz / (8 * g.M)));
        h->tzc = (g.Nz + nchunk - 1) / nchunk;
    } else {
        int nchunk = std::max(1, (g.Nz + 56) / 112);
        h->tzc = (g.Nz + nchunk - 1) / nchunk;
    }
    h->src_scale = (float)(d3 ? cfg->dt / (cfg->dz * cfg->dy * cfg->dx) : cfg->dt / (cfg->dz * cfg->dx));

    // model on the device
    CHECK(dalloc_t(h, &h->scratch1, 2 * h->nint));
    const float *vp_d, *rho_d;
    CHECK(stage_in(h, vp, h->scratch1, h->nint, &vp_d));
    CHECK(stage_in(h, rho, h->scratch1 + h->nint, h->nint, &rho_d));
    CHECK(dalloc_t(h, &h->flag, 4));
    CHECK(check_finite(h, vp_d, h->nint, "vp"));
    CHECK(check_finite(h, rho_d, h->nint, "rho"));
    CHECK(dalloc_t(h, &h->fscal, 8));
    double vmax = cfg->pml_vmax;
    if (!(vmax > 0)) {
        CU(launch_max_abs_reduce(vp_d, h->nint, h->fscal, h->work));
        float vm = 0.f;
        CU(cudaMemcpyAsync(&vm, h->fscal, sizeof(float), cudaMemcpyDeviceToHost, h->work));
        CU(cudaStreamSynchronize(h->work));
        vmax = vm;
    }
    {
        double s = 0.0, inv2 = 1.0 / (cfg->dz * cfg->dz) + 1.0 / (cfg->dx * cfg->dx);
        if (d3) inv2 += 1.0 / (cfg->dy * cfg->dy);
        for (int l = 0; l < g.M; ++l) s += std::fabs(c[l]);
        double lim = 1.0 / (vmax * std::sqrt(inv2) * s);
        if (!(cfg->dt < lim)) {
            char buf[160];
            std::snprintf(buf, sizeof buf, "dt = %g exceeds the stability limit %g", cfg->dt, lim);
            return fail(LSRTM_ERR_CFL, buf);
        }
    }
    CHECK(dalloc_t(h, &h->kdt, 2 * g.plane));   // (kdt, binv) adjacent: one tensor map covers both
    h->binv = h->kdt + g.plane;
    CHECK(dalloc_t(h, &h->kd2, 2 * g.plane));   // (kd2, br2) adjacent: one tensor map covers both
    h->br2 = h->kd2 + g.plane;
    CU(launch_model_prep(g, vp_d, rho_d, h->kdt, h->binv, h->work));
    h->launches++;
    h->gm = g;
    CHECK(setup_windows(h, geo));

    // CPML profiles: per direction ai bi ah bh
    {
        int N[3] = {g.Nz, g.Ny, g.Nx};
        int o[3] = {g.z0, g.y0, g.x0};
        int ni[3] = {g.nz, g.ny, g.nx};
        double hh[3] = {cfg->dz, cfg->dy, cfg->dx};
        size_t tot = 4 * ((size_t)N[0] + N[1] + N[2]);
        std::vector<float> prof(tot, 0.f);
        CHECK(dalloc_t(h, &h->pml_buf, tot));
        size_t off = 0;
        for (int d = 0; d < 3; ++d) {
            float *b = prof.data() + off;
            if (!(d == 1 && g.ndim == 2))
                cpml_profile(N[d], o[d], ni[d], cfg->npml, hh[d], vmax, cfg->f0, cfg->dt, b, b + N[d],
                             b + 2 * N[d], b + 3 * N[d]);
            if (d == 0 && g.fs)   // no CPML above a free surface (nodes and half nodes above row z0)
                for (int i = 0; i < o[0]; ++i) b[i] = b[N[d] + i] = b[2 * N[d] + i] = b[3 * N[d] + i] = 0.f;
            h->pml.ai[d] = h->pml_buf + off;
            h->pml.bi[d] = h->pml_buf + off + N[d];
            h->pml.ah[d] = h->pml_buf + off + 2 * N[d];
            h->pml.bh[d] = h->pml_buf + off + 3 * N[d];
            off += 4 * (size_t)N[d];
        }
        CU(cudaMemcpyAsync(h->pml_buf, prof.data(), tot * sizeof(float), cudaMemcpyHostToDevice, h->work));
        CU(cudaStreamSynchronize(h->work));
    }
    if (h->win) {
        // x profiles of every shot's own window: [4][nshot][Nx] (ai, bi, ah, bh)
        const int nwin = (int)h->win_nx_h.size();
        const size_t stride = (size_t)g.Nx, per = (size_t)nwin * stride;
        std::vector<float> prof(4 * per, 0.f);
        for (int s = 0; s < nwin; ++s) {
            float *b = prof.data() + (size_t)s * stride;
            cpml_profile(h->win_nx_h[s] + 2 * g.x0, g.x0, h->win_nx_h[s], cfg->npml, cfg->dx, vmax, cfg->f0,
                         cfg->dt, b, b + per, b + 2 * per, b + 3 * per);
        }
        float *px;
        CHECK(dalloc_t(h, &px, 4 * per));
        CU(cudaMemcpyAsync(px, prof.data(), 4 * per * sizeof(float), cudaMemcpyHostToDevice, h->work));
        CU(cudaStreamSynchronize(h->work));
        h->pml.ai[2] = px;
        h->pml.bi[2] = px + per;
        h->pml.ah[2] = px + 2 * per;
        h->pml.bh[2] = px + 3 * per;
    }

    CHECK(build_geometry(h, geo));
    size_t nw = (size_t)(cfg->wavelet_per_shot ? h->nshot : 1) * g.nt;
    CHECK(dalloc_t(h, &h->wav, nw));
    CU(cudaMemcpyAsync(h->wav, wavelet, nw * sizeof(float), cudaMemcpyDefault, h->work));

    // staging and Krylov vectors
    long long nd = h->nrec_total * g.nt;
    CHECK(dalloc_t(h, &h->dstage, std::max<long long>(nd, 1)));
    CHECK(dalloc_t(h, &h->mstage, 2 * h->nint));
    CHECK(dalloc_t(h, &h->gstage, 2 * h->nint));
    CHECK(dalloc_t(h, &h->img_acc, h->nint));
    CHECK(dalloc_t(h, &h->hess_acc, h->nint));
    CHECK(dalloc_t(h, &h->hess_img, h->nint));
    CHECK(dalloc_t(h, &h->scal, 16));
    {
        const double one = 1.0;
        CU(cudaMemcpyAsync(h->scal + 5, &one, sizeof(double), cudaMemcpyHostToDevice, h->work));
        CU(cudaStreamSynchronize(h->work));
    }
    CHECK(dalloc_t(h, &h->dotwork, 152 * 4 + 32));

    // Reconstruction of the background in reverse time: boundary bands of
    // every shot over all nt steps (cached across L^T calls), or, when those do
    // not fit, full-state checkpoints every K steps per batch from which the
    // bands of one K-step segment at a time are recomputed.
    h->bands.nb = d3 ? 2LL * g.M * ((long long)g.nz * g.ny + (long long)g.nz * g.nx + (long long)g.ny * g.nx)
                     : 2LL * g.M * (g.nz + g.nx);
    h->bands.fmt = cfg->plan == LSRTM_PLAN_PLAIN ? BAND_F32
                   : (cfg->band_precision == LSRTM_BAND_BF16 ? BAND_BF16S
                                                              : (cfg->band_precision == LSRTM_BAND_FP16 ? BAND_F16S : BAND_F32));
    const size_t esz = h->bands.fmt == BAND_F32 ? 4 : 2;
    const size_t fbytes = (size_t)g.plane * sizeof(float);
    h->fs_planes = d3 ? 4 : 3;

    // wavefield slots
    // 2D: ping-pong state + in-place node CPML planes + image plane; 3D: one in-place state
    // of 20 planes (pairs, CPML memories, images) + the pseudo-Hessian plane
    h->sstride = (d3 ? kStatePlanes3D : (h->win ? kWinStatePlanes2D : kStatePlanes2D)) * g.plane;
    h->vstride = d3 ? 0 : kPsivPlanes2D * g.plane;
    // 3D: st[0] (20 planes; the fused kernels use its first 14 as ping and the
    // last 6 as the in-place node CPML memories), st[1] (14 planes, pong), the
    // float2 image plane and the pseudo-Hessian plane
    h->sstride1 = d3 ? 2LL * kBornPairs3F * g.plane : h->sstride;
    if (h->sstride >= (1LL << 31))   // the time-step kernels index within a slot with 32-bit offsets
        return fail(LSRTM_ERR_ARG, "grid too large: a wavefield slot exceeds 2^31 floats");
    size_t per_slot = d3 ? ((size_t)h->sstride + h->sstride1 + 3 * g.plane) * sizeof(float)
                         : (2 * (size_t)h->sstride + h->vstride + 2 * g.plane + g.plane) * sizeof(float);
    if (h->bands.fmt != BAND_F32) per_slot += 2 * (size_t)h->bands.nb * sizeof(float);   // FP32 band stage
    int batch = cfg->plan == LSRTM_PLAN_PLAIN ? 1 : (cfg->shots_per_batch > 0 ? cfg->shots_per_batch : h->nshot);
    batch = std::min(batch, h->nshot);
    size_t cg_bytes = (5 * 2 * (size_t)h->nint + (size_t)nd) * sizeof(float);
    long long avail;   // bytes left for bands, checkpoints and slots
    if (cfg->hbm_budget_bytes) {
        avail = (long long)cfg->hbm_budget_bytes - (long long)h->bytes - (long long)cg_bytes;
    } else {
        size_t fr = 0, tot = 0;
        CU(cudaMemGetInfo(&fr, &tot));
        avail = (long long)(0.92 * (double)fr) - (long long)cg_bytes;
    }
    const size_t band_full = 2 * (size_t)h->nshot * g.nt * h->bands.nb * esz;
    const size_t scale_full = h->bands.fmt != BAND_F32 ? 2 * (size_t)h->nshot * g.nt * sizeof(float) : 0;
    const size_t fs_full = (size_t)h->nshot * h->fs_planes * fbytes;
    bool ckpt = cfg->recon_mode == LSRTM_RECON_CHECKPOINT;
    if (cfg->recon_mode == LSRTM_RECON_AUTO)
        ckpt = !h->win && (long long)(band_full + scale_full + fs_full + per_slot) > avail;
    if (ckpt && h->win)
        return fail(LSRTM_ERR_ARG, "checkpoint reconstruction does not support aperture windows");
    h->ckpt = ckpt;
    if (!ckpt) {
        CHECK(dalloc(h, &h->band_mem, band_full));
        h->bands.p = h->band_mem;
        h->bands.v = static_cast<char *>(h->band_mem) + band_full / 2;
        h->bands.shot0 = 0;
        h->bands.t0 = 0;
        h->bands.nsteps = g.nt;
        if (h->bands.fmt != BAND_F32) CHECK(dalloc_t(h, &h->bands.scale, (size_t)h->nshot * g.nt * 2));
        CHECK(dalloc_t(h, &h->final_state, (size_t)h->nshot * h->fs_planes * g.plane));
        avail -= (long long)(band_full + scale_full + fs_full);
    } else {
        // checkpoint: the background planes of a forward state (2D: p vx vz psi_px
        // psi_pz + the two node CPML memories; 3D: p, v, psi_p, psi_v)
        h->ck_planes = d3 ? 10 : 7;
        h->ck_fmt = cfg->plan == LSRTM_PLAN_PLAIN ? BAND_F32
                    : (cfg->checkpoint_precision == LSRTM_BAND_BF16 ? BAND_BF16S
                                                                    : (cfg->checkpoint_precision == LSRTM_BAND_FP16
                                                                           ? BAND_F16S
                                                                           : BAND_F32));
        const double seg_step = 2.0 * (double)h->bands.nb * esz;           // band bytes per step
        const double ck_one = (double)h->ck_planes * g.plane * ck_esize(h) + h->ck_planes * sizeof(float);
        int K = cfg->checkpoint_interval > 0
                    ? cfg->checkpoint_interval
                    : (int)std::lround(std::sqrt((double)g.nt * ck_one / seg_step));
        K = std::max(1, std::min(K, g.nt));
        h->ck_K = K;
        h->ck_nseg = (g.nt + K - 1) / K;
        // recomputation state: 2D 5 + 5 ping-pong planes and 2 CPML planes; 3D 10 in place
        size_t rec_slot = (d3 ? 10 : 12) * fbytes;
        size_t ck_slot = (size_t)h->ck_nseg * (size_t)ck_one + (size_t)K * (size_t)seg_step +
                         rec_slot + h->fs_planes * fbytes +
                         (h->bands.fmt != BAND_F32 ? 2 * (size_t)K * sizeof(float) : 0);
        per_slot += ck_slot;
    }
    if (avail < (long long)per_slot)
        return fail(LSRTM_ERR_OOM, cfg->hbm_budget_bytes ? "hbm_budget_bytes too small for one wavefield slot"
                                                         : "device memory too small for one wavefield slot");
    {
        long long fit = avail / (long long)per_slot;
        if (fit < batch) batch = (int)fit;
    }
    h->batch = batch;
    if (ckpt) {
        const size_t segb = (size_t)batch * h->ck_K * h->bands.nb * esz;
        CHECK(dalloc(h, &h->band_mem, 2 * segb));
        h->segbands = h->bands;
        h->segbands.p = h->band_mem;
        h->segbands.v = static_cast<char *>(h->band_mem) + segb;
        h->segbands.nsteps = h->ck_K;
        if (h->segbands.fmt != BAND_F32) CHECK(dalloc_t(h, &h->segbands.scale, (size_t)batch * h->ck_K * 2));
        h->bands = h->segbands;
        h->bands.shot0 = 0;
        h->bands.t0 = 0;
        CHECK(dalloc(h, &h->ck_mem, (size_t)h->ck_nseg * batch * h->ck_planes * g.plane * ck_esize(h)));
        if (h->ck_fmt != BAND_F32) CHECK(dalloc_t(h, &h->ck_amax, (size_t)h->ck_nseg * batch * h->ck_planes));
        CHECK(dalloc_t(h, &h->final_state, (size_t)batch * h->fs_planes * g.plane));
        if (d3) {
            CHECK(dalloc_t(h, &h->rec[0], (size_t)batch * 10 * g.plane));
        } else {
            CHECK(dalloc_t(h, &h->rec[0], (size_t)batch * 5 * g.plane));
            CHECK(dalloc_t(h, &h->rec[1], (size_t)batch * 5 * g.plane));
            CHECK(dalloc_t(h, &h->rec_psiv, (size_t)batch * 2 * g.plane));
        }
    }
    if (h->bands.fmt != BAND_F32) {
        CHECK(dalloc_t(h, &h->bands.stage, (size_t)batch * 2 * h->bands.nb));
        h->segbands.stage = h->bands.stage;
    }
    CHECK(dalloc_t(h, &h->st[0], (size_t)batch * h->sstride));
    CHECK(dalloc_t(h, &h->st[1], (size_t)batch * h->sstride1));
    if (!d3) CHECK(dalloc_t(h, &h->psiv, (size_t)batch * h->vstride));
    CHECK(dalloc_t(h, &h->img, (size_t)batch * g.plane));
    CHECK(dalloc_t(h, &h->hess, (size_t)batch * g.plane));
    CHECK(dalloc_t(h, &h->kerr, 4));
    h->guard_K = cfg->guard_interval < 0 ? 0 : (cfg->guard_interval ? cfg->guard_interval : kGuardInterval);
    h->g.abort = h->kerr + 1;
    CU(cudaMallocHost(reinterpret_cast<void **>(&h->poll_h), 4 * sizeof(int)));
    for (cudaEvent_t &e : h->poll_ev) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (d3) CHECK(setup_fused3d(h));
    else if (!h->win) {
        for (int b = 0; b < 2; ++b) {
            cudaError_t e = maps2d(&h->m2d[b], h->g, h->st[b], h->sstride, h->kdt, h->binv, h->kd2, h->br2, h->img,
                                   batch);
            if (e != cudaSuccess) return fail(LSRTM_ERR_CUDA, std::string("tensor maps: ") + cudaGetErrorString(e));
        }
        h->tma2d = true;
    }
    CU(cudaStreamSynchronize(h->work));
    return LSRTM_OK;
}

lsrtm_status ensure_cg(lsrtm_handle *h)
{
    if (h->cg_x) return LSRTM_OK;
    size_t m = 2 * (size_t)h->nint;
    CHECK(dalloc_t(h, &h->cg_x, m));
    CHECK(dalloc_t(h, &h->cg_s, m));
    CHECK(dalloc_t(h, &h->cg_z, m));
    CHECK(dalloc_t(h, &h->cg_p, m));
    CHECK(dalloc_t(h, &h->cg_minv, m));
    CHECK(dalloc_t(h, &h->cg_r, std::max<long long>(h->nrec_total * h->g.nt, 1)));
    return LSRTM_OK;
}

}  // namespace

extern "C" {

lsrtm_status lsrtm_create(const lsrtm_config *cfg, const float *vp, const float *rho,
                          const float *wavelet, const lsrtm_geometry *geom, void *stream,
                          lsrtm_handle **out)
{
    g_last_error.clear();
    if (!out || !vp || !rho || !wavelet) return fail(LSRTM_ERR_ARG, "null argument");
    *out = nullptr;
    lsrtm_handle *h = new (std::nothrow) lsrtm_handle();
    if (!h) return fail(LSRTM_ERR_OOM, "host allocation failed");
    lsrtm_status s = create_impl(cfg, vp, rho, wavelet, geom, stream, h);
    if (s != LSRTM_OK) {
        std::string msg = g_last_error;
        lsrtm_destroy(h);
        g_last_error = msg;
        return s;
    }
    *out = h;
    return LSRTM_OK;
}

lsrtm_status lsrtm_born(lsrtm_handle *h, const float *dm, float *d)
{
    if (!h || !dm || !d) return fail(LSRTM_ERR_ARG, "null argument");
    CHECK(begin_call(h));
    const float *dm_d;
    CHECK(stage_in(h, dm, h->mstage, 2 * h->nint, &dm_d));
    CHECK(prep_perturbation(h, dm_d));
    CHECK(born_core(h));
    CHECK(copy_out(h, d, h->dstage, h->nrec_total * h->g.nt));
    return end_call(h, !is_device_ptr(d));
}

lsrtm_status lsrtm_adjoint(lsrtm_handle *h, const float *d, float *g, float *pseudo_hess)
{
    if (!h || !d || !g) return fail(LSRTM_ERR_ARG, "null argument");
    CHECK(begin_call(h));
    CHECK(copy_out(h, h->dstage, d, h->nrec_total * h->g.nt));
    bool gdev = is_device_ptr(g);
    float *gd = gdev ? g : h->gstage;
    CHECK(adjoint_core(h, gd, pseudo_hess != nullptr));
    if (!gdev) CHECK(copy_out(h, g, gd, 2 * h->nint));
    bool hdev = true;
    if (pseudo_hess) {
        hdev = is_device_ptr(pseudo_hess);
        CHECK(copy_out(h, pseudo_hess, h->hess_img, h->nint));
    }
    return end_call(h, !gdev || !hdev);
}

lsrtm_status lsrtm_model(lsrtm_handle *h, float *d)
{
    if (!h || !d) return fail(LSRTM_ERR_ARG, "null argument");
    CHECK(begin_call(h));
    CHECK(model_core(h));
    CHECK(copy_out(h, d, h->dstage, h->nrec_total * h->g.nt));
    return end_call(h, !is_device_ptr(d));
}

lsrtm_status lsrtm_mute_residual(lsrtm_handle *h, const float *d_obs, const float *d_syn, double v_mute, double t0,
                                 double t_taper, double o_max, double o_taper, float *d_out)
{
    if (!h || !d_obs || !d_out) return fail(LSRTM_ERR_ARG, "null argument");
    if (!(v_mute > 0.0) || !(t_taper >= 0.0) || !(o_taper >= 0.0) || !std::isfinite(t0) || !std::isfinite(o_max))
        return fail(LSRTM_ERR_ARG, "v_mute must be > 0, the tapers >= 0 and t0, o_max finite");
    const long long nrec = h->nrec_total, nt = h->g.nt, nd = nrec * nt;
    CHECK(begin_call(h));
    if (!h->mute_n0) {
        CHECK(dalloc_t(h, &h->mute_n0, std::max<long long>(nrec, 1)));
        CHECK(dalloc_t(h, &h->mute_a0, std::max<long long>(nrec, 1)));
        CHECK(dalloc_t(h, &h->mute_fo, std::max<long long>(nrec, 1)));
    }
    // per receiver, in FP64: the mute time td = o / v_mute + t0, the first
    // sample n0 with t_n = (n + 1) dt past it, (t_n0 - td) / t_taper, and the
    // far-offset factor
    const double dt = h->cfg.dt;
    std::vector<int> n0(nrec);
    std::vector<float> a0(nrec), fo(nrec);
    for (long long r = 0; r < nrec; ++r) {
        const double o = h->rec_off_h[r];
        const double td = o / v_mute + t0;
        const double q = td / dt;
        long long n;
        if (!(q < (double)nt + 1.0)) {
            n = nt;   // the mute time is past the record (or not finite): every sample muted
        } else {
            n = q > 1.0 ? (long long)std::floor(q) - 1 : 0;   // then the first n with (n + 1) dt - td > 0
            while (n < nt && (n + 1) * dt - td <= 0.0) ++n;
            while (n > 0 && n * dt - td > 0.0) --n;
        }
        n0[r] = (int)std::min<long long>(n, nt);
        a0[r] = t_taper > 0.0 ? (float)(((n0[r] + 1) * dt - td) / t_taper) : 0.f;
        double f = 1.0;
        if (o_max > 0.0) {
            const double u = o_max - o;
            if (u <= 0.0) f = 0.0;
            else if (o_taper > 0.0 && u < o_taper) f = 0.5 * (1.0 - std::cos(3.14159265358979323846 * u / o_taper));
        }
        fo[r] = (float)f;
    }
    if (nrec > 0) {
        CU(cudaMemcpyAsync(h->mute_n0, n0.data(), nrec * sizeof(int), cudaMemcpyHostToDevice, h->work));
        CU(cudaMemcpyAsync(h->mute_a0, a0.data(), nrec * sizeof(float), cudaMemcpyHostToDevice, h->work));
        CU(cudaMemcpyAsync(h->mute_fo, fo.data(), nrec * sizeof(float), cudaMemcpyHostToDevice, h->work));
    }
    const float *a, *b = nullptr;
    CHECK(stage_in(h, d_obs, h->dstage, nd, &a));
    if (d_syn) {
        if (!is_device_ptr(d_syn) && !h->dstage2) CHECK(dalloc_t(h, &h->dstage2, std::max<long long>(nd, 1)));
        CHECK(stage_in(h, d_syn, h->dstage2, nd, &b));
    }
    const bool odev = is_device_ptr(d_out);
    float *od = odev ? d_out : h->dstage;
    CU(launch_mute_residual(a, b, h->mute_n0, h->mute_a0, h->mute_fo, nrec, (int)nt,
                            t_taper > 0.0 ? (float)(dt / t_taper) : 0.f, od, h->work));
    h->launches++;
    if (!odev) CHECK(copy_out(h, d_out, od, nd));
    // the host vectors must outlive the queued copies
    return end_call(h, true);
}

lsrtm_status lsrtm_remigrate(lsrtm_handle *h, const float *m, float *out)
{
    if (!h || !m || !out) return fail(LSRTM_ERR_ARG, "null argument");
    CHECK(begin_call(h));
    const float *m_d;
    CHECK(stage_in(h, m, h->mstage, 2 * h->nint, &m_d));
    CHECK(prep_perturbation(h, m_d));
    CHECK(born_core(h));
    bool odev = is_device_ptr(out);
    float *od = odev ? out : h->gstage;
    CHECK(adjoint_core(h, od, false));
    if (!odev) CHECK(copy_out(h, out, od, 2 * h->nint));
    return end_call(h, !odev);
}

lsrtm_status lsrtm_psf(lsrtm_handle *h, int param, int spacing, float *psf)
{
    if (!h || !psf) return fail(LSRTM_ERR_ARG, "null argument");
    if (param != 0 && param != 1) return fail(LSRTM_ERR_ARG, "param must be 0 (Vp) or 1 (Ip)");
    if (spacing < 1) return fail(LSRTM_ERR_ARG, "spacing must be >= 1");
    CHECK(begin_call(h));
    CU(launch_comb(h->gm, param, spacing, h->mstage, h->work));
    h->launches++;
    CHECK(prep_perturbation(h, h->mstage));
    CHECK(born_core(h));
    bool odev = is_device_ptr(psf);
    float *od = odev ? psf : h->gstage;
    CHECK(adjoint_core(h, od, false));
    if (!odev) CHECK(copy_out(h, psf, od, 2 * h->nint));
    return end_call(h, !odev);
}

}  // extern "C"

namespace {

// CGNR (CGLS form), Sec. 3, with FP64 device scalars:
//   begin:   x = P x0, r = d - L x, s = P L^T r, z = M^-1 s, p = z, gamma = <s, z>
//   iterate: q = L p, alpha = gamma / <q, q>, x += alpha p, r -= alpha q,
//            s = P L^T r, z = M^-1 s, gamma' = <s, z>, p = z + (gamma'/gamma) p
// P zeroes the planes outside param_mask; M is the diagonal pseudo-Hessian.
lsrtm_status cg_begin_impl(lsrtm_handle *h, const float *d, const float *x0, int precond,
                           int param_mask)
{
    CHECK(ensure_cg(h));
    const long long nm = 2 * h->nint;
    const long long nd = h->nrec_total * h->g.nt;
    cudaStream_t s = h->work;
    double *gamma = h->scal + 0, *dd = h->scal + 3, *one = h->scal + 5;
    h->cg_mask = param_mask;
    h->cg_precond = precond;
    h->cg_iter = 0;
    if (x0) CHECK(copy_out(h, h->cg_x, x0, nm));
    else CU(cudaMemsetAsync(h->cg_x, 0, nm * sizeof(float), s));
    CU(launch_mul_mask(h->cg_x, nullptr, param_mask, h->nint, s));
    CHECK(copy_out(h, h->cg_r, d, nd));
    CU(launch_dot(h->cg_r, h->cg_r, nd, dd, h->dotwork, s));
    h->launches += 3;
    if (x0) {
        CHECK(prep_perturbation(h, h->cg_x));
        CHECK(born_core(h));
        CU(launch_axpy_ratio(h->cg_r, h->dstage, one, one, -1.0f, nd, s));
        h->launches++;
    }
    if (precond) {
        if (!h->hess_ready) CHECK(h->ckpt ? ck_hessian(h) : bg_forward(h, true));
        CU(cudaMemsetAsync(h->fscal, 0, sizeof(float), s));
        CU(launch_max_abs_reduce(h->hess_img, h->nint, h->fscal, s));
        CU(launch_precond_build(h->hess_img, h->fscal, 1e-3f, h->nint, h->cg_minv, s));
        h->launches += 2;
    }
    CU(launch_scale_copy(h->dstage, h->cg_r, nd, s));
    CHECK(adjoint_core(h, h->cg_s, false));
    CU(launch_mul_mask(h->cg_s, nullptr, param_mask, h->nint, s));
    CU(launch_scale_copy(h->cg_z, h->cg_s, nm, s));
    if (precond) CU(launch_mul_mask(h->cg_z, h->cg_minv, param_mask, h->nint, s));
    CU(launch_scale_copy(h->cg_p, h->cg_z, nm, s));
    CU(launch_dot(h->cg_s, h->cg_z, nm, gamma, h->dotwork, s));
    CU(launch_dot(h->cg_r, h->cg_r, nd, h->scal + 6, h->dotwork, s));
    // gamma_new and <q,q> of an earlier solve are not this solve's: clear them
    // before the guard reads the scalars
    CU(cudaMemsetAsync(h->scal + 1, 0, 2 * sizeof(double), s));
    CU(launch_guard_scalars(h->scal, 7, h->kerr + 1, guard_code(GK_CG, 0), s));
    h->launches += 11;
    h->cg_active = true;
    return LSRTM_OK;
}

lsrtm_status cg_iterate_impl(lsrtm_handle *h, int niter)
{
    const long long nm = 2 * h->nint;
    const long long nd = h->nrec_total * h->g.nt;
    cudaStream_t s = h->work;
    double *gamma = h->scal + 0, *gnew = h->scal + 1, *qq = h->scal + 2;
    if (h->mis_cap < h->cg_iter + niter + 1) {
        int cap = std::max(2 * (h->cg_iter + niter + 1), 64);
        double *nb = nullptr;
        CHECK(dalloc_t(h, &nb, cap));
        if (h->mis_dev) CU(cudaMemcpyAsync(nb, h->mis_dev, h->mis_cap * sizeof(double), cudaMemcpyDeviceToDevice, s));
        h->mis_dev = nb;
        h->mis_cap = cap;
    }
    for (int k = 0; k < niter; ++k) {
        CHECK(prep_perturbation(h, h->cg_p));
        CHECK(born_core(h));
        CU(launch_dot(h->dstage, h->dstage, nd, qq, h->dotwork, s));
        CU(launch_axpy_ratio(h->cg_x, h->cg_p, gamma, qq, 1.0f, nm, s));
        CU(launch_axpy_ratio(h->cg_r, h->dstage, gamma, qq, -1.0f, nd, s));
        CU(launch_scale_copy(h->dstage, h->cg_r, nd, s));
        CHECK(adjoint_core(h, h->cg_s, false));
        CU(launch_mul_mask(h->cg_s, nullptr, h->cg_mask, h->nint, s));
        CU(launch_scale_copy(h->cg_z, h->cg_s, nm, s));
        if (h->cg_precond) CU(launch_mul_mask(h->cg_z, h->cg_minv, h->cg_mask, h->nint, s));
        CU(launch_dot(h->cg_s, h->cg_z, nm, gnew, h->dotwork, s));
        CU(launch_xpby_ratio(h->cg_p, h->cg_z, gnew, gamma, nm, s));
        CU(cudaMemcpyAsync(gamma, gnew, sizeof(double), cudaMemcpyDeviceToDevice, s));
        h->cg_iter++;
        CU(launch_dot(h->cg_r, h->cg_r, nd, h->mis_dev + h->cg_iter, h->dotwork, s));
        // the iteration's FP64 scalars: <q,q>, gamma, <d,d> and <r,r>
        CU(launch_guard_scalars(h->scal, 7, h->kerr + 1, guard_code(GK_CG, h->cg_iter), s));
        CU(launch_guard_scalars(h->mis_dev + h->cg_iter, 1, h->kerr + 1, guard_code(GK_CG, h->cg_iter), s));
        h->launches += 18;
        // Poll the error words without draining the queue: copy this
        // iteration's words to pinned memory, then wait for the copy of the
        // previous iteration while this one runs. A tripped guard ends the
        // solve here (the queued iteration's time loops return at once).
        int *ph = h->poll_h + 2 * (k & 1);
        CU(cudaMemcpyAsync(ph, h->kerr, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaEventRecord(h->poll_ev[k & 1], s));
        if (k > 0) {
            const int j = (k - 1) & 1;
            CU(cudaEventSynchronize(h->poll_ev[j]));
            if (h->poll_h[2 * j] || h->poll_h[2 * j + 1]) return check_kernel_error(h);
        }
    }
    return LSRTM_OK;
}

lsrtm_status read_misfits(lsrtm_handle *h, int first, int count, double *out)
{
    std::vector<double> m2(count);
    double dd = 0.0;
    CU(cudaMemcpyAsync(m2.data(), h->mis_dev + first, count * sizeof(double), cudaMemcpyDeviceToHost, h->work));
    CU(cudaMemcpyAsync(&dd, h->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, h->work));
    CU(cudaStreamSynchronize(h->work));
    for (int k = 0; k < count; ++k) out[k] = dd > 0 ? std::sqrt(m2[k] / dd) : 0.0;
    return LSRTM_OK;
}

}  // namespace

extern "C" {

lsrtm_status lsrtm_cg_begin(lsrtm_handle *h, const float *d, const float *x0, int precond,
                            int param_mask)
{
    if (!h || !d) return fail(LSRTM_ERR_ARG, "null argument");
    if (param_mask < 1 || param_mask > 3) return fail(LSRTM_ERR_ARG, "param_mask must be 1, 2 or 3");
    CHECK(begin_call(h));
    h->cg_active = false;
    CHECK(cg_begin_impl(h, d, x0, precond, param_mask));
    if (h->mis_cap < 64) {
        CHECK(dalloc_t(h, &h->mis_dev, 64));
        h->mis_cap = 64;
    }
    CU(cudaMemcpyAsync(h->mis_dev, h->scal + 6, sizeof(double), cudaMemcpyDeviceToDevice, h->work));
    return end_call(h, false);
}

lsrtm_status lsrtm_cg_iterate(lsrtm_handle *h, int niter, double *misfit)
{
    if (!h) return fail(LSRTM_ERR_ARG, "null handle");
    if (!h->cg_active) return fail(LSRTM_ERR_STATE, "lsrtm_cg_begin has not been called");
    if (niter < 0) return fail(LSRTM_ERR_ARG, "niter < 0");
    CHECK(begin_call(h));
    int first = h->cg_iter + 1;
    CHECK(cg_iterate_impl(h, niter));
    CHECK(end_call(h, misfit != nullptr));   // reading the misfits synchronises anyway
    if (misfit && niter > 0) CHECK(read_misfits(h, first, niter, misfit));
    return LSRTM_OK;
}

lsrtm_status lsrtm_cg_get_state(lsrtm_handle *h, float *x, float *p, float *r, double *scalars, int *iter)
{
    if (!h || !x || !p || !r || !scalars || !iter) return fail(LSRTM_ERR_ARG, "null argument");
    if (!h->cg_active) return fail(LSRTM_ERR_STATE, "lsrtm_cg_begin has not been called");
    CHECK(begin_call(h));
    const long long nm = 2 * h->nint, nd = h->nrec_total * h->g.nt;
    CHECK(copy_out(h, x, h->cg_x, nm));
    CHECK(copy_out(h, p, h->cg_p, nm));
    CHECK(copy_out(h, r, h->cg_r, nd));
    double sc[2] = {0.0, 0.0};
    CU(cudaMemcpyAsync(&sc[0], h->scal + 0, sizeof(double), cudaMemcpyDeviceToHost, h->work));
    CU(cudaMemcpyAsync(&sc[1], h->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, h->work));
    CHECK(end_call(h, true));
    CU(cudaMemcpy(scalars, sc, sizeof(sc), cudaMemcpyDefault));
    *iter = h->cg_iter;
    return LSRTM_OK;
}

lsrtm_status lsrtm_cg_set_state(lsrtm_handle *h, const float *x, const float *p, const float *r,
                                const double *scalars, int iter)
{
    if (!h || !x || !p || !r || !scalars) return fail(LSRTM_ERR_ARG, "null argument");
    if (iter < 0) return fail(LSRTM_ERR_ARG, "iteration count < 0");
    if (!h->cg_active) return fail(LSRTM_ERR_STATE, "lsrtm_cg_begin has not been called");
    CHECK(begin_call(h));
    const long long nm = 2 * h->nint, nd = h->nrec_total * h->g.nt;
    double sc[2];
    CU(cudaMemcpy(sc, scalars, sizeof(sc), cudaMemcpyDefault));
    if (h->mis_cap < iter + 1) {
        const int cap = std::max(2 * (iter + 1), 64);
        double *nb = nullptr;
        CHECK(dalloc_t(h, &nb, cap));
        if (h->mis_dev) CU(cudaMemcpyAsync(nb, h->mis_dev, h->mis_cap * sizeof(double), cudaMemcpyDeviceToDevice,
                                           h->work));
        h->mis_dev = nb;
        h->mis_cap = cap;
    }
    CHECK(copy_out(h, h->cg_x, x, nm));
    CHECK(copy_out(h, h->cg_p, p, nm));
    CHECK(copy_out(h, h->cg_r, r, nd));
    CU(cudaMemcpyAsync(h->scal + 0, &sc[0], sizeof(double), cudaMemcpyHostToDevice, h->work));
    CU(cudaMemcpyAsync(h->scal + 3, &sc[1], sizeof(double), cudaMemcpyHostToDevice, h->work));
    CU(launch_dot(h->cg_r, h->cg_r, nd, h->mis_dev + iter, h->dotwork, h->work));   // <r, r> of that iterate
    h->launches++;
    h->cg_iter = iter;
    // the host copies of the scalars must outlive the queued copies
    return end_call(h, true);
}

lsrtm_status lsrtm_cg_result(lsrtm_handle *h, float *dm, double *misfit0)
{
    if (!h || !dm) return fail(LSRTM_ERR_ARG, "null argument");
    if (!h->cg_active) return fail(LSRTM_ERR_STATE, "lsrtm_cg_begin has not been called");
    CHECK(begin_call(h));
    CHECK(copy_out(h, dm, h->cg_x, 2 * h->nint));
    CHECK(end_call(h, true));
    if (misfit0) CHECK(read_misfits(h, 0, 1, misfit0));
    return check_finite(h, h->cg_x, 2 * h->nint, "CG solution");
}

lsrtm_status lsrtm_cg_solve(lsrtm_handle *h, const float *d, float *dm, int niter, int precond,
                            int param_mask, double *misfit)
{
    if (!h || !d || !dm) return fail(LSRTM_ERR_ARG, "null argument");
    if (niter < 0) return fail(LSRTM_ERR_ARG, "niter < 0");
    CHECK(lsrtm_cg_begin(h, d, dm, precond, param_mask));
    CHECK(lsrtm_cg_iterate(h, niter, misfit ? misfit + 1 : nullptr));
    return lsrtm_cg_result(h, dm, misfit);
}

lsrtm_status lsrtm_timing_enable(lsrtm_handle *h, int enable)
{
    if (!h) return fail(LSRTM_ERR_ARG, "null handle");
    h->timing = enable != 0;
    return LSRTM_OK;
}

lsrtm_status lsrtm_timing_read(lsrtm_handle *h, lsrtm_timings *out, int reset)
{
    if (!h || !out) return fail(LSRTM_ERR_ARG, "null argument");
    CU(cudaStreamSynchronize(h->work));
    for (auto &t : h->pending) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, t.a, t.b));
        h->t_ms[t.kind] += ms;
        h->t_launch[t.kind] += t.launches;
        h->t_cells[t.kind] += t.cells;
        h->event_pool.push_back(t.a);
        h->event_pool.push_back(t.b);
    }
    h->pending.clear();
    out->born_ms = h->t_ms[0];
    out->background_ms = h->t_ms[1];
    out->adjoint_ms = h->t_ms[2];
    out->born_launches = h->t_launch[0];
    out->background_launches = h->t_launch[1];
    out->adjoint_launches = h->t_launch[2];
    out->born_cells = h->t_cells[0];
    out->background_cells = h->t_cells[1];
    out->adjoint_cells = h->t_cells[2];
    if (reset)
        for (int k = 0; k < 3; ++k) h->t_ms[k] = 0, h->t_launch[k] = 0, h->t_cells[k] = 0;
    return LSRTM_OK;
}

lsrtm_status lsrtm_set_stream(lsrtm_handle *h, void *stream)
{
    if (!h) return fail(LSRTM_ERR_ARG, "null handle");
    h->user = (cudaStream_t)stream;
    return LSRTM_OK;
}

lsrtm_status lsrtm_deblur(lsrtm_handle *h, const float *m_rtm, const float *m_remig, int spacing, int flen,
                          double eps, float *dm_out, float *filters)
{
    if (!h || !m_rtm || !m_remig || !dm_out) return fail(LSRTM_ERR_ARG, "null argument");
    if (h->g.ndim != 2) return fail(LSRTM_ERR_ARG, "lsrtm_deblur supports 2D images only");
    if (flen < 1 || flen > 11 || flen % 2 == 0) return fail(LSRTM_ERR_ARG, "flen must be odd and in [1, 11]");
    if (spacing < 2 || spacing > 48) return fail(LSRTM_ERR_ARG, "spacing must be in [2, 48]");
    if (!(eps >= 0.0)) return fail(LSRTM_ERR_ARG, "eps must be >= 0");
    const int nz = h->gm.nz, nx = h->gm.nx;   // the model grid (the slot grid is the widest window)
    if (nz <= spacing / 2 || nx <= spacing / 2)
        return fail(LSRTM_ERR_ARG, "image smaller than half the node spacing: no deblurring node");
    const int nkz = deblur_nodes(nz, spacing), nkx = deblur_nodes(nx, spacing);
    const size_t nf = 2 * (size_t)nkz * nkx * flen * flen;
    CHECK(begin_call(h));
    if (nf > h->db_cap) {
        CHECK(dalloc_t(h, &h->db_filt, nf));
        h->db_cap = nf;
    }
    if (!h->db_out) CHECK(dalloc_t(h, &h->db_out, 2 * (size_t)h->nint));
    const float *a, *b;
    CHECK(stage_in(h, m_rtm, h->mstage, 2 * h->nint, &a));
    CHECK(stage_in(h, m_remig, h->gstage, 2 * h->nint, &b));
    CU(cudaMemsetAsync(h->flag, 0, sizeof(int), h->work));
    const bool odev = is_device_ptr(dm_out);
    float *od = odev ? dm_out : h->db_out;
    CU(launch_deblur(a, b, nz, nx, spacing, flen, eps, h->db_filt, od, h->flag, h->work));
    h->launches += 2;
    if (!odev) CHECK(copy_out(h, dm_out, od, 2 * h->nint));
    if (filters) CHECK(copy_out(h, filters, h->db_filt, nf));
    int flag = 0;
    CU(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->work));
    CHECK(end_call(h, true));
    if (flag) return fail(LSRTM_ERR_NONFINITE, "deblurring normal equations not positive definite (eps too small "
                                              "or non-finite images); those filters are set to zero");
    return LSRTM_OK;
}

lsrtm_status lsrtm_deblur_wiener(lsrtm_handle *h, const float *m_rtm, const float *m_remig, int spacing, double eps,
                                 float *dm_out)
{
    if (!h || !m_rtm || !m_remig || !dm_out) return fail(LSRTM_ERR_ARG, "null argument");
    if (h->g.ndim != 2) return fail(LSRTM_ERR_ARG, "lsrtm_deblur_wiener supports 2D images only");
    if (spacing < 2 || spacing > wiener_max_spacing()) return fail(LSRTM_ERR_ARG, "spacing must be in [2, 32]");
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail(LSRTM_ERR_ARG, "eps must be > 0");
    const int nz = h->gm.nz, nx = h->gm.nx;
    if (nz <= spacing / 2 || nx <= spacing / 2)
        return fail(LSRTM_ERR_ARG, "image smaller than half the node spacing: no deblurring node");
    const int nkz = deblur_nodes(nz, spacing), nkx = deblur_nodes(nx, spacing);
    const size_t nb = 2 * (size_t)nkz * nkx * 4 * spacing * spacing;
    CHECK(begin_call(h));
    if (nb > h->wn_cap) {
        CHECK(dalloc_t(h, &h->wn_blk, nb));
        h->wn_cap = nb;
    }
    if (!h->db_out) CHECK(dalloc_t(h, &h->db_out, 2 * (size_t)h->nint));
    const float *a, *b;
    CHECK(stage_in(h, m_rtm, h->mstage, 2 * h->nint, &a));
    CHECK(stage_in(h, m_remig, h->gstage, 2 * h->nint, &b));
    const bool odev = is_device_ptr(dm_out);
    float *od = odev ? dm_out : h->db_out;
    CU(launch_wiener(a, b, nz, nx, spacing, eps, h->wn_blk, od, h->work));
    h->launches += 2;
    if (!odev) CHECK(copy_out(h, dm_out, od, 2 * h->nint));
    return end_call(h, !odev);
}

}  // extern "C"

namespace {

// The interpolated PSF Hessian of one call: 2D or 3D arguments of the kernels.
struct PsfhPlan {
    bool d3 = false;
    PsfHessDev a2{};
    PsfHess3Dev a3{};
};

cudaError_t psfh_apply(const PsfhPlan &pl, bool transpose, const float *in, float *out, cudaStream_t s)
{
    return pl.d3 ? launch_psfh3_apply(pl.a3, transpose, in, out, s) : launch_psfh_apply(pl.a2, transpose, in, out, s);
}

// Validates the PSF Hessian arguments, stages the PSF images and builds the
// node windows; the caller has called begin_call.
lsrtm_status psfh_setup(lsrtm_handle *h, const float *psf_vp, const float *psf_ip, int spacing, int half,
                        int param_mask, PsfhPlan *pl)
{
    const bool d3 = h->g.ndim == 3;
    if (param_mask < 1 || param_mask > 3) return fail(LSRTM_ERR_ARG, "param_mask must be 1, 2 or 3");
    if (spacing < 2 || spacing > 64) return fail(LSRTM_ERR_ARG, "spacing must be in [2, 64]");
    if (half < 0) half = (spacing - 1) / 2;
    if (half > kPsfHessMaxHalf) return fail(LSRTM_ERR_ARG, "half must be <= 15");
    if ((param_mask & 1) && !psf_vp) return fail(LSRTM_ERR_ARG, "param_mask includes Vp but psf_vp is NULL");
    if ((param_mask & 2) && !psf_ip) return fail(LSRTM_ERR_ARG, "param_mask includes Ip but psf_ip is NULL");
    const int nz = h->gm.nz, ny = h->gm.ny, nx = h->gm.nx;
    if (nz <= spacing / 2 || nx <= spacing / 2 || (d3 && ny <= spacing / 2))
        return fail(LSRTM_ERR_ARG, "image smaller than half the node spacing: no comb node");
    if (d3 && nz > 65535) return fail(LSRTM_ERR_ARG, "3D PSF Hessian: nz must be <= 65535");
    const int nkz = deblur_nodes(nz, spacing), nkx = deblur_nodes(nx, spacing);
    const int nky = d3 ? deblur_nodes(ny, spacing) : 1;
    const long long L = 2 * half + 1;
    const long long npt = (long long)nkz * nky * nkx * L * L * (d3 ? L : 1);
    if (npt >= (1LL << 31)) return fail(LSRTM_ERR_ARG, "too many node windows for this spacing and half");
    const size_t m = 2 * (size_t)h->nint;
    if (!h->ph_vec) CHECK(dalloc_t(h, &h->ph_vec, 8 * m));
    if (!h->ph_scal) CHECK(dalloc_t(h, &h->ph_scal, 8));
    if ((size_t)npt > h->ph_cap) {
        CHECK(dalloc_t(h, &h->ph_pt, (size_t)npt));
        h->ph_cap = (size_t)npt;
    }
    const float *pv = nullptr, *pi = nullptr;
    if (param_mask & 1) CHECK(stage_in(h, psf_vp, h->ph_vec + 6 * m, m, &pv));
    if (param_mask & 2) CHECK(stage_in(h, psf_ip, h->ph_vec + 7 * m, m, &pi));
    pl->d3 = d3;
    if (d3) {
        pl->a3 = PsfHess3Dev{nz, ny, nx, spacing, half, nkz, nky, nkx, param_mask, h->ph_pt};
        CU(launch_psfh3_patches(pv, pi, pl->a3, h->ph_pt, h->work));
    } else {
        pl->a2 = PsfHessDev{nz, nx, spacing, half, nkz, nkx, param_mask, h->ph_pt};
        CU(launch_psfh_patches(pv, pi, nz, nx, spacing, half, nkz, nkx, param_mask, h->ph_pt, h->work));
    }
    h->launches++;
    return LSRTM_OK;
}

}  // namespace

extern "C" {

lsrtm_status lsrtm_psf_hessian(lsrtm_handle *h, const float *psf_vp, const float *psf_ip, int spacing, int half,
                               int param_mask, int transpose, const float *x, float *y)
{
    if (!h || !x || !y) return fail(LSRTM_ERR_ARG, "null argument");
    if ((const void *)x == (const void *)y) return fail(LSRTM_ERR_ARG, "x and y must not overlap");
    CHECK(begin_call(h));
    PsfhPlan a;
    CHECK(psfh_setup(h, psf_vp, psf_ip, spacing, half, param_mask, &a));
    const size_t m = 2 * (size_t)h->nint;
    const float *xd;
    CHECK(stage_in(h, x, h->ph_vec + 5 * m, m, &xd));
    const bool odev = is_device_ptr(y);
    float *od = odev ? y : h->ph_vec + 4 * m;
    CU(psfh_apply(a, transpose != 0, xd, od, h->work));
    h->launches++;
    if (!odev) CHECK(copy_out(h, y, od, m));
    return end_call(h, !odev);
}

// CGNR (CGLS form) on H^H H dm = H^H P m_rtm from dm = 0, FP64 device scalars:
//   r = P m_rtm, s = H^T r, p = s, gamma = <s, s>; per iteration
//   q = H p, alpha = gamma / <q, q>, dm += alpha p, r -= alpha q,
//   s = H^T r, gamma' = <s, s>, p = s + (gamma'/gamma) p.
lsrtm_status lsrtm_psf_cg(lsrtm_handle *h, const float *psf_vp, const float *psf_ip, int spacing, int half,
                          int param_mask, const float *m_rtm, float *dm, int niter, double *misfit)
{
    if (!h || !m_rtm || !dm) return fail(LSRTM_ERR_ARG, "null argument");
    if (niter < 0) return fail(LSRTM_ERR_ARG, "niter < 0");
    CHECK(begin_call(h));
    PsfhPlan a;
    CHECK(psfh_setup(h, psf_vp, psf_ip, spacing, half, param_mask, &a));
    const long long m = 2 * h->nint;
    float *v = h->ph_vec;
    float *X = v, *R = v + m, *S = v + 2 * m, *Pp = v + 3 * m, *Q = v + 4 * m;
    const float *md;
    CHECK(stage_in(h, m_rtm, v + 5 * m, m, &md));
    if (h->ph_mis_cap < niter + 1) {
        const int cap = std::max(niter + 1, 64);
        CHECK(dalloc_t(h, &h->ph_mis, cap));
        h->ph_mis_cap = cap;
    }
    cudaStream_t s = h->work;
    double *gamma = h->ph_scal, *gnew = h->ph_scal + 1, *qq = h->ph_scal + 2, *dd = h->ph_scal + 3;
    CU(cudaMemsetAsync(X, 0, m * sizeof(float), s));
    CU(launch_scale_copy(R, md, m, s));
    CU(launch_mul_mask(R, nullptr, param_mask, h->nint, s));
    CU(launch_dot(R, R, m, dd, h->dotwork, s));
    CU(psfh_apply(a, true, R, S, s));
    CU(launch_scale_copy(Pp, S, m, s));
    CU(launch_dot(S, S, m, gamma, h->dotwork, s));
    CU(cudaMemcpyAsync(h->ph_mis, dd, sizeof(double), cudaMemcpyDeviceToDevice, s));
    h->launches += 6;
    for (int k = 0; k < niter; ++k) {
        CU(psfh_apply(a, false, Pp, Q, s));
        CU(launch_dot(Q, Q, m, qq, h->dotwork, s));
        CU(launch_axpy_ratio(X, Pp, gamma, qq, 1.0f, m, s));
        CU(launch_axpy_ratio(R, Q, gamma, qq, -1.0f, m, s));
        CU(psfh_apply(a, true, R, S, s));
        CU(launch_dot(S, S, m, gnew, h->dotwork, s));
        CU(launch_xpby_ratio(Pp, S, gnew, gamma, m, s));
        CU(cudaMemcpyAsync(gamma, gnew, sizeof(double), cudaMemcpyDeviceToDevice, s));
        CU(launch_dot(R, R, m, h->ph_mis + k + 1, h->dotwork, s));
        h->launches += 8;
    }
    CHECK(copy_out(h, dm, X, m));
    std::vector<double> m2(niter + 1);
    double d2 = 0.0;
    CU(cudaMemcpyAsync(m2.data(), h->ph_mis, (niter + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(&d2, dd, sizeof(double), cudaMemcpyDeviceToHost, s));
    CHECK(end_call(h, true));
    if (misfit)
        for (int k = 0; k <= niter; ++k) misfit[k] = d2 > 0 ? std::sqrt(m2[k] / d2) : 0.0;
    return check_finite(h, X, m, "PSF-Hessian CG solution");
}

lsrtm_status lsrtm_autotune(lsrtm_handle *h, int steps, int *tzc_out, double *ms_out, int *ncand_out)
{
    if (!h) return fail(LSRTM_ERR_ARG, "null handle");
    CHECK(begin_call(h));
    const bool d3 = is3d(h);
    const GridDev &g = h->g;
    // candidates: the padded depth split into 1..12 chunks of at least 2M + 8 rows
    std::vector<int> cand;
    for (int nchunk = 1; nchunk <= 12; ++nchunk) {
        int t = (g.Nz + nchunk - 1) / nchunk;
        if (t < 2 * g.M + 8) break;
        if (cand.empty() || cand.back() != t) cand.push_back(t);
    }
    if (std::find(cand.begin(), cand.end(), h->tzc) == cand.end()) cand.push_back(h->tzc);
    int maxsteps = g.nt - 1;
    if (h->ckpt) maxsteps = std::min(maxsteps, h->ck_K);
    steps = std::max(1, std::min(steps > 0 ? steps : 16, maxsteps));
    const int bs = batch_size(h, 0);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    double best = 1e300;
    int best_tzc = h->tzc;
    std::vector<double> times;
    lsrtm_status st = LSRTM_OK;
    for (int c : cand) {
        h->tzc = c;
        if ((st = build_tiles(h)) != LSRTM_OK) break;
        if ((st = zero_slots(h, bs)) != LSRTM_OK) break;
        if ((st = gather_model(h, 0, bs, true)) != LSRTM_OK) break;
        Step2D a = step_args(h, 0);
        double ms = 0.0;
        for (int rep = 0; rep < 2 && st == LSRTM_OK; ++rep) {   // first pass warms up
            cudaEventRecord(e0, h->work);
            for (int i = 0; i < steps; ++i) {
                if (d3) {
                    Step3F &b = h->f3born[i & 1];
                    b.n = i;
                    b.shot0 = 0;
                    b.trec = h->trv;
                    b.tzc = c;
                    launch_born3f(b, bs, h->work);
                    adj3f_step(h, i, steps - i, 0, h->bands);
                    continue;
                }
                a.n = i;
                a.in = h->st[i & 1];
                a.out = h->st[(i + 1) & 1];
                launch_fwd2d(a, bs, true, false, false, h->work, maps2_of(h, i & 1));
                a.n = steps - i;
                launch_adj2d(a, maps2_of(h, i & 1), bs, h->work);
            }
            cudaEventRecord(e1, h->work);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) st = fail(LSRTM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
            float f = 0.f;
            cudaEventElapsedTime(&f, e0, e1);
            ms = f / steps;
        }
        h->launches += 4LL * steps;
        times.push_back(ms);
        if (d3 && st == LSRTM_OK) st = check_kernel_error(h);   // a fused kernel's wait that gave up
        if (st != LSRTM_OK) break;
        if (ms < best) {
            best = ms;
            best_tzc = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->tzc = best_tzc;
    lsrtm_status s2 = build_tiles(h);
    if (st == LSRTM_OK) st = s2;
    // graphs captured with the previous chunking are stale
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    h->graph_guards.clear();
    h->bg_cached = false;
    if (st != LSRTM_OK) return st;
    if (tzc_out) *tzc_out = best_tzc;
    if (ncand_out) *ncand_out = (int)cand.size();
    if (ms_out)
        for (size_t i = 0; i < times.size(); ++i) {
            ms_out[2 * i] = cand[i];
            ms_out[2 * i + 1] = times[i];
        }
    return end_call(h, true);
}

lsrtm_status lsrtm_reconstruction(const lsrtm_handle *h, int *mode, int *interval, int *batch)
{
    if (!h) return fail(LSRTM_ERR_ARG, "null handle");
    if (mode) *mode = h->ckpt ? LSRTM_RECON_CHECKPOINT : LSRTM_RECON_BOUNDARY;
    if (interval) *interval = h->ckpt ? h->ck_K : 0;
    if (batch) *batch = h->batch;
    return LSRTM_OK;
}

lsrtm_status lsrtm_synchronize(lsrtm_handle *h)
{
    if (!h) return fail(LSRTM_ERR_ARG, "null handle");
    CU(cudaStreamSynchronize(h->work));
    CU(cudaGetLastError());
    return check_kernel_error(h);
}

size_t lsrtm_workspace_bytes(const lsrtm_handle *h) { return h ? h->bytes : 0; }

long long lsrtm_kernel_launches(const lsrtm_handle *h) { return h ? h->launches : 0; }

void lsrtm_destroy(lsrtm_handle *h)
{
    if (!h) return;
    if (h->work) cudaStreamSynchronize(h->work);
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    for (auto &t : h->pending) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
    for (void *p : h->allocs) cudaFree(p);
    if (h->poll_h) cudaFreeHost(h->poll_h);
    for (cudaEvent_t e : h->poll_ev)
        if (e) cudaEventDestroy(e);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->work) cudaStreamDestroy(h->work);
    delete h;
}

const char *lsrtm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace lsrtm {
// Lets other translation units of the library report through lsrtm_last_error.
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace lsrtm
