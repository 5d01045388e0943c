// Host runtime and C ABI of libbh (declared in include/bh.h): model object,
// C-PML profiles, shot plan, forward-history store, and the drivers that
// enqueue the kernels of bh_kernels.cuh / bh_ops.cuh on the model's stream.
#include "bh.h"
#include "bh_kernels.cuh"
#include "bh_ops.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace bh;

namespace {

thread_local std::string g_create_error;

struct ShotDev {
    int z0 = 0, nz = 0, src_ir = 0, src_iz = 0, nrec = 0;
    std::vector<int> rec_iz;
    int* d_recmap = nullptr;                       // [nz]
    float* d_zprof = nullptr;                      // az_int, bz_int, az_half, bz_half [4][nz]
    float* d_hist = nullptr;                       // [nt][2][nr*P]
};

}  // namespace

struct bh_model {
    bh_grid_desc grid{};
    int nzg = 0, nshots = 0, nrec_max = 0, P = 0;
    cudaStream_t stream = nullptr;
    double vpmax = 0.0;
    // model, global [nr][nzg]
    float *d_lam = nullptr, *d_mu = nullptr, *d_rho = nullptr;
    float *d_bvr = nullptr, *d_bvz = nullptr, *d_muh = nullptr;
    uint8_t* d_mask = nullptr;
    uint8_t* d_colcov = nullptr;
    // radial profiles: inv_r_int, inv_r_half, ar_int, br_int, ar_half, br_half [6][nr]
    float* d_rprof = nullptr;
    std::vector<ShotDev> shots;
    // working state of one window
    float* d_state = nullptr;   // 6 fields [nr*P]
    float* d_psi = nullptr;     // 16 planes [nr*P]: 8 memories x 2 (ping-pong)
    float2* d_G = nullptr;      // 5 Kahan planes [nr*P]
    float* d_H = nullptr;       // 3 planes [nr*P]
    double* d_Hg = nullptr;     // H_lam, H_mu global [2][nr*nzg]
    double* d_scal = nullptr;   // small device scalars
    bool have_forward = false, have_gradient = false;
    std::string err;
    // persistent (one cooperative launch per shot and direction) or one
    // launch per half-step; co-resident blocks of the persistent kernels
    int persistent = 1;
    int fwd_blocks = 0, adj_blocks = 0;
    unsigned* d_bar = nullptr;          // barrier: count, generation, error flag
    double barrier_timeout_ms = 2000.0;
    int barrier_extra = 0;              // test knob: arrivals that never come
    // sampled kernel timing: events around every prof_every-th step's launches
    int prof_every = 0;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, size_t>> prof_marks;  // (kernel id, first event index)
    double prof_ms[BH_KERNEL_COUNT] = {0};
    long prof_n[BH_KERNEL_COUNT] = {0};
};

namespace {

bh_status fail(bh_model* m, bh_status s, const std::string& msg)
{
    if (m) m->err = msg;
    else g_create_error = msg;
    return s;
}

#define BH_CUDA(m, call)                                                                 \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail((m), e_ == cudaErrorMemoryAllocation ? BH_ERR_OOM : BH_ERR_CUDA, \
                        std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)

#define BH_LAUNCH(m)                                                                      \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess)                                                            \
            return fail((m), BH_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc((void**)p, count * sizeof(T));
}

void free_model(bh_model* m)
{
    if (!m) return;
    cudaFree(m->d_lam);
    cudaFree(m->d_mu);
    cudaFree(m->d_rho);
    cudaFree(m->d_bvr);
    cudaFree(m->d_bvz);
    cudaFree(m->d_muh);
    cudaFree(m->d_mask);
    cudaFree(m->d_colcov);
    cudaFree(m->d_rprof);
    for (auto& s : m->shots) {
        cudaFree(s.d_recmap);
        cudaFree(s.d_zprof);
        cudaFree(s.d_hist);
    }
    cudaFree(m->d_state);
    cudaFree(m->d_psi);
    cudaFree(m->d_G);
    cudaFree(m->d_H);
    cudaFree(m->d_Hg);
    cudaFree(m->d_scal);
    cudaFree(m->d_bar);
    for (cudaEvent_t e : m->ev_pool) cudaEventDestroy(e);
    delete m;
}

// C-PML coefficients (recursive convolution, kappa = 1) at depth fraction x
void pml_ab(double x, double d0, double alpha_max, double dt, double* a, double* b)
{
    x = std::min(1.0, std::max(0.0, x));
    double d = d0 * x * x;
    double alpha = alpha_max * (1.0 - x);
    *b = std::exp(-(d + alpha) * dt);
    *a = d > 0.0 ? d * (*b - 1.0) / (d + alpha) : 0.0;
}

size_t nrp(const bh_model* m) { return (size_t)m->grid.nr * m->P; }

WinK make_win(const bh_model* m, const ShotDev& s)
{
    WinK g;
    g.nr = m->grid.nr;
    g.nz = s.nz;
    g.P = m->P;
    g.nzg = m->nzg;
    g.z0 = s.z0;
    g.npml_r = m->grid.npml_r;
    g.npml_z = m->grid.npml_z;
    g.dt = (float)m->grid.dt;
    g.inv_dr = (float)(1.0 / m->grid.dr);
    g.inv_dz = (float)(1.0 / m->grid.dz);
    return g;
}

CoefK make_coef(const bh_model* m, const ShotDev& s)
{
    const int nr = m->grid.nr;
    CoefK C;
    C.lam = m->d_lam;
    C.mu = m->d_mu;
    C.rho = m->d_rho;
    C.bvr = m->d_bvr;
    C.bvz = m->d_bvz;
    C.muh = m->d_muh;
    C.inv_r_int = m->d_rprof;
    C.inv_r_half = m->d_rprof + nr;
    C.ar_int = m->d_rprof + 2 * nr;
    C.br_int = m->d_rprof + 3 * nr;
    C.ar_half = m->d_rprof + 4 * nr;
    C.br_half = m->d_rprof + 5 * nr;
    C.az_int = s.d_zprof;
    C.bz_int = s.d_zprof + s.nz;
    C.az_half = s.d_zprof + 2 * s.nz;
    C.bz_half = s.d_zprof + 3 * s.nz;
    return C;
}

StateK make_state(const bh_model* m, int parity)
{
    const size_t n = nrp(m);
    StateK S;
    S.vr = m->d_state;
    S.vz = m->d_state + n;
    S.trr = m->d_state + 2 * n;
    S.ttt = m->d_state + 3 * n;
    S.tzz = m->d_state + 4 * n;
    S.trz = m->d_state + 5 * n;
    for (int k = 0; k < 8; ++k) {
        float* a = m->d_psi + (size_t)k * n;
        float* b = m->d_psi + (size_t)(8 + k) * n;
        if (parity < 0) {          // forward: update in place in bank a
            S.psi[k] = S.psi_w[k] = a;
        } else {                   // adjoint: read one bank, write the other
            S.psi[k] = parity ? b : a;
            S.psi_w[k] = parity ? a : b;
        }
    }
    return S;
}

// Sampled timing of one kernel launch: returns the event index to close, or
// SIZE_MAX when this launch is not sampled.
size_t prof_begin(bh_model* m, int kernel, int step)
{
    if (m->prof_every <= 0 || step % m->prof_every != 0) return SIZE_MAX;
    if (m->ev_used + 2 > m->ev_pool.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return SIZE_MAX;
            m->ev_pool.push_back(e);
        }
    }
    size_t i = m->ev_used;
    m->ev_used += 2;
    cudaEventRecord(m->ev_pool[i], m->stream);
    m->prof_marks.push_back({kernel, i});
    return i;
}

void prof_end(bh_model* m, size_t i)
{
    if (i != SIZE_MAX) cudaEventRecord(m->ev_pool[i + 1], m->stream);
}

dim3 block2d() { return dim3(32, 8); }
dim3 grid2d(int nr, int nz) { return dim3((nz + 31) / 32, (nr + 7) / 8); }
// grid of the tiled stepping kernels: one block per kTR x kTZ tile
int n_tiles(int nr, int nz) { return ((nz + kTZ - 1) / kTZ) * ((nr + kTR - 1) / kTR); }
dim3 grid_tiles(int nr, int nz) { return dim3(n_tiles(nr, nz)); }

BarK make_bar(const bh_model* m, int blocks)
{
    BarK b;
    b.count = m->d_bar;
    b.err = (int*)(m->d_bar + 2);
    b.expected = (unsigned)blocks + (unsigned)m->barrier_extra;
    b.timeout_ns = (unsigned long long)(m->barrier_timeout_ms * 1e6);
    return b;
}

// Read the barrier error flag of the last persistent launch (synchronises).
bh_status check_barrier(bh_model* m)
{
    int err = 0;
    BH_CUDA(m, cudaMemcpyAsync(&err, m->d_bar + 2, sizeof(int), cudaMemcpyDeviceToHost,
                               m->stream));
    BH_CUDA(m, cudaStreamSynchronize(m->stream));
    if (err)
        return fail(m, BH_ERR_TIMEOUT,
                    "a grid barrier of the persistent stepping kernel timed out; results are invalid");
    return BH_OK;
}

// Launch a stepping kernel with programmatic stream serialization: its
// blocks may be scheduled while the previous kernel drains and wait in
// griddepcontrol.wait for its results.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t stream,
                       Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

bh_status rebuild_coefficients(bh_model* m)
{
    const int nr = m->grid.nr, nzg = m->nzg;
    k_setup_nodes<<<grid2d(nr, nzg), block2d(), 0, m->stream>>>(nr, nzg, m->d_mu, m->d_rho,
                                                                m->d_bvr, m->d_bvz, m->d_muh);
    BH_LAUNCH(m);
    return BH_OK;
}

bh_status load_model(bh_model* m, const float* vp, const float* vs, const float* rho,
                     bool first)
{
    const int nr = m->grid.nr, nzg = m->nzg;
    const size_t n = (size_t)nr * nzg;
    // CFL check and C-PML d0 need max Vp
    k_max_f32<<<1, kRedThreads, 0, m->stream>>>(n, vp, m->d_scal);
    BH_LAUNCH(m);
    double vpmax = 0.0;
    BH_CUDA(m, cudaMemcpyAsync(&vpmax, m->d_scal, sizeof(double), cudaMemcpyDeviceToHost,
                               m->stream));
    BH_CUDA(m, cudaStreamSynchronize(m->stream));
    if (!(vpmax > 0.0) || !std::isfinite(vpmax))
        return fail(m, BH_ERR_INVALID_ARG, "vp must be positive and finite");
    const bh_grid_desc& g = m->grid;
    const double cfl = g.dt * vpmax * std::sqrt(1.0 / (g.dr * g.dr) + 1.0 / (g.dz * g.dz)) *
                       (9.0 / 8.0 + 1.0 / 24.0);
    if (cfl >= 1.0) {
        char buf[160];
        snprintf(buf, sizeof buf, "CFL number %.4f >= 1 (dt %.3g s, max Vp %.1f m/s)", cfl, g.dt,
                 vpmax);
        return fail(m, BH_ERR_CFL, buf);
    }
    // the C-PML profiles keep the max Vp of the model given at creation
    if (first) m->vpmax = vpmax;
    const int tpb = 256;
    k_setup_cells<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, m->stream>>>((int)n, vp, vs, rho,
                                                                         m->d_lam, m->d_mu,
                                                                         m->d_rho);
    BH_LAUNCH(m);
    if (first) {
        k_setup_mask<<<grid2d(nr, nzg), block2d(), 0, m->stream>>>(nr, nzg, g.npml_r, vs,
                                                                   m->d_colcov, m->d_mask);
        BH_LAUNCH(m);
    }
    bh_status st = rebuild_coefficients(m);
    if (st != BH_OK) return st;
    m->have_forward = m->have_gradient = false;
    return BH_OK;
}

bh_status setup_profiles(bh_model* m)
{
    const bh_grid_desc& g = m->grid;
    const int nr = g.nr;
    const double alpha_max = M_PI * g.f0;
    const double R = g.pml_R > 0.0 ? g.pml_R : 1e-3;
    std::vector<float> rp(6 * (size_t)nr);
    const double Lr = g.npml_r * g.dr;
    const double d0r = g.npml_r > 0 ? -3.0 * m->vpmax * std::log(R) / (2.0 * Lr) : 0.0;
    for (int i = 0; i < nr; ++i) {
        double ri = i * g.dr, rh = (i + 0.5) * g.dr;
        rp[i] = i > 0 ? (float)(1.0 / ri) : 0.f;
        rp[nr + i] = (float)(1.0 / rh);
        double a, b;
        double xi = g.npml_r > 0 ? (ri - (nr - g.npml_r) * g.dr) / Lr : 0.0;
        double xh = g.npml_r > 0 ? (rh - (nr - g.npml_r) * g.dr) / Lr : 0.0;
        pml_ab(xi, d0r, alpha_max, g.dt, &a, &b);
        rp[2 * nr + i] = (float)a;
        rp[3 * nr + i] = (float)b;
        pml_ab(xh, d0r, alpha_max, g.dt, &a, &b);
        rp[4 * nr + i] = (float)a;
        rp[5 * nr + i] = (float)b;
    }
    BH_CUDA(m, cudaMemcpyAsync(m->d_rprof, rp.data(), rp.size() * sizeof(float),
                               cudaMemcpyHostToDevice, m->stream));
    const double Lz = g.npml_z * g.dz;
    const double d0z = g.npml_z > 0 ? -3.0 * m->vpmax * std::log(R) / (2.0 * Lz) : 0.0;
    for (auto& s : m->shots) {
        const int nz = s.nz;
        std::vector<float> zp(4 * (size_t)nz);
        for (int j = 0; j < nz; ++j)
            for (int h = 0; h < 2; ++h) {
                double z = (j + 0.5 * h) * g.dz, x = 0.0;
                if (g.npml_z > 0) {
                    double xt = ((g.npml_z - 0.5) * g.dz - z) / Lz;
                    double xb = (z - (nz - g.npml_z - 0.5) * g.dz) / Lz;
                    x = std::max(xt, xb);
                }
                double a, b;
                pml_ab(x, d0z, alpha_max, g.dt, &a, &b);
                zp[(2 * h) * nz + j] = (float)a;
                zp[(2 * h + 1) * nz + j] = (float)b;
            }
        BH_CUDA(m, cudaMemcpyAsync(s.d_zprof, zp.data(), zp.size() * sizeof(float),
                                   cudaMemcpyHostToDevice, m->stream));
        std::vector<int> recmap(nz, -1);
        for (int k = 0; k < s.nrec; ++k) recmap[s.rec_iz[k]] = k;
        BH_CUDA(m, cudaMemcpyAsync(s.d_recmap, recmap.data(), nz * sizeof(int),
                                   cudaMemcpyHostToDevice, m->stream));
        // host vectors must outlive the copies
        BH_CUDA(m, cudaStreamSynchronize(m->stream));
    }
    return BH_OK;
}

}  // namespace

// error text of calls that have no model (read with bh_last_error(NULL))
void bh_internal_set_thread_error(const std::string& msg) { g_create_error = msg; }

extern "C" {

const char* bh_status_string(bh_status s)
{
    switch (s) {
    case BH_OK: return "ok";
    case BH_ERR_INVALID_ARG: return "invalid argument";
    case BH_ERR_CFL: return "CFL condition violated";
    case BH_ERR_OOM: return "out of device memory";
    case BH_ERR_CUDA: return "CUDA error";
    case BH_ERR_TIMEOUT: return "device wait timed out";
    case BH_ERR_STATE: return "call out of order";
    case BH_ERR_UNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

const char* bh_last_error(const bh_model* m)
{
    return m ? m->err.c_str() : g_create_error.c_str();
}

bh_status bh_model_create(const bh_grid_desc* grid, int nz_global, const float* vp,
                          const float* vs, const float* rho, const bh_shot_desc* shots,
                          int nshots, void* stream, bh_model** out)
{
    g_create_error.clear();
    if (!out) return fail(nullptr, BH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !vp || !vs || !rho || !shots || nshots <= 0)
        return fail(nullptr, BH_ERR_INVALID_ARG, "NULL argument or nshots <= 0");
    const bh_grid_desc& g = *grid;
    if (g.nr < 4 || nz_global < 4 || g.nt < 1 || g.npml_r < 0 || g.npml_z < 0 ||
        g.nr - g.npml_r < 4 || !(g.dr > 0) || !(g.dz > 0) || !(g.dt > 0) || g.f0 < 0 ||
        g.nz != nz_global)
        return fail(nullptr, BH_ERR_INVALID_ARG, "bad grid description");
    if (g.snapshot_precision != 0)
        return fail(nullptr, BH_ERR_UNSUPPORTED, "reduced-precision history not built");
    if (g.checkpoint_cap_bytes != 0)
        return fail(nullptr, BH_ERR_UNSUPPORTED, "checkpointed history not built");
    int nzmax = 0, nrec_max = 0;
    for (int s = 0; s < nshots; ++s) {
        const bh_shot_desc& d = shots[s];
        if (d.nz < 4 || d.z_offset < 0 || d.z_offset + d.nz > nz_global || 2 * g.npml_z >= d.nz)
            return fail(nullptr, BH_ERR_INVALID_ARG, "shot window outside the model");
        if (d.src_ir < 0 || d.src_ir >= g.nr - g.npml_r || d.src_iz < g.npml_z ||
            d.src_iz >= d.nz - g.npml_z)
            return fail(nullptr, BH_ERR_INVALID_ARG, "source outside the window interior");
        if (d.nrec < 0 || (d.nrec > 0 && !d.rec_iz))
            return fail(nullptr, BH_ERR_INVALID_ARG, "bad receiver list");
        for (int k = 0; k < d.nrec; ++k)
            if (d.rec_iz[k] < g.npml_z || d.rec_iz[k] >= d.nz - g.npml_z)
                return fail(nullptr, BH_ERR_INVALID_ARG, "receiver outside the window interior");
        nzmax = std::max(nzmax, d.nz);
        nrec_max = std::max(nrec_max, d.nrec);
    }

    bh_model* m = new bh_model();
    m->grid = g;
    m->nzg = nz_global;
    m->nshots = nshots;
    m->nrec_max = nrec_max;
    m->P = (nzmax + 31) / 32 * 32;
    m->stream = (cudaStream_t)stream;
    const int nr = g.nr;
    const size_t ng = (size_t)nr * nz_global;
    const size_t nw = (size_t)nr * m->P;

    auto bail = [&](bh_status s) {
        g_create_error = m->err;
        free_model(m);
        return s;
    };
#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            m->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
            return bail(e_ == cudaErrorMemoryAllocation ? BH_ERR_OOM : BH_ERR_CUDA);    \
        }                                                                               \
    } while (0)
    CK(dalloc(&m->d_lam, ng));
    CK(dalloc(&m->d_mu, ng));
    CK(dalloc(&m->d_rho, ng));
    CK(dalloc(&m->d_bvr, ng));
    CK(dalloc(&m->d_bvz, ng));
    CK(dalloc(&m->d_muh, ng));
    CK(dalloc(&m->d_mask, ng));
    CK(dalloc(&m->d_colcov, (size_t)nz_global));
    CK(dalloc(&m->d_rprof, 6 * (size_t)nr));
    CK(dalloc(&m->d_state, 6 * nw));
    CK(dalloc(&m->d_psi, 16 * nw));
    CK(dalloc(&m->d_G, 5 * nw));
    CK(dalloc(&m->d_H, 3 * nw));
    CK(dalloc(&m->d_Hg, 2 * ng));
    CK(dalloc(&m->d_scal, 16));
    CK(dalloc(&m->d_bar, 4));
    {
        int dev = 0, sms = 0, coop = 0, nb = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fwd_persist, kThreads, 0));
        m->fwd_blocks = nb * sms;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_persist, kThreads, 0));
        m->adj_blocks = nb * sms;
        if (!coop || m->fwd_blocks < 1 || m->adj_blocks < 1) m->persistent = 0;
    }
    m->shots.resize(nshots);
    std::vector<uint8_t> colcov(nz_global, 0);
    for (int s = 0; s < nshots; ++s) {
        ShotDev& sd = m->shots[s];
        const bh_shot_desc& d = shots[s];
        sd.z0 = d.z_offset;
        sd.nz = d.nz;
        sd.src_ir = d.src_ir;
        sd.src_iz = d.src_iz;
        sd.nrec = d.nrec;
        sd.rec_iz.assign(d.rec_iz, d.rec_iz + d.nrec);
        for (int j = g.npml_z; j < d.nz - g.npml_z; ++j) colcov[d.z_offset + j] = 1;
        CK(dalloc(&sd.d_recmap, (size_t)d.nz));
        CK(dalloc(&sd.d_zprof, 4 * (size_t)d.nz));
        CK(dalloc(&sd.d_hist, (size_t)g.nt * 2 * nw));
    }
    CK(cudaMemcpyAsync(m->d_colcov, colcov.data(), nz_global, cudaMemcpyHostToDevice,
                       m->stream));
    CK(cudaMemsetAsync(m->d_psi, 0, 16 * nw * sizeof(float), m->stream));
    CK(cudaStreamSynchronize(m->stream));
#undef CK
    bh_status st = load_model(m, vp, vs, rho, true);
    if (st != BH_OK) return bail(st);
    st = setup_profiles(m);
    if (st != BH_OK) return bail(st);
    *out = m;
    return BH_OK;
}

void bh_model_destroy(bh_model* m)
{
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    free_model(m);
}

bh_status bh_set_model(bh_model* m, const float* vp, const float* vs, const float* rho)
{
    if (!m || !vp || !vs || !rho) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    return load_model(m, vp, vs, rho, false);
}

bh_status bh_forward(bh_model* m, const float* wavelet, float* seis)
{
    if (!m || !wavelet || !seis) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    const bh_grid_desc& gd = m->grid;
    const size_t nw = nrp(m);
    const size_t seis_per_shot = (size_t)m->nrec_max * gd.nt;
    BH_CUDA(m, cudaMemsetAsync(seis, 0, seis_per_shot * m->nshots * sizeof(float), m->stream));
    for (int s = 0; s < m->nshots; ++s) {
        ShotDev& sd = m->shots[s];
        WinK g = make_win(m, sd);
        CoefK C = make_coef(m, sd);
        StateK S = make_state(m, -1);
        BH_CUDA(m, cudaMemsetAsync(m->d_state, 0, 6 * nw * sizeof(float), m->stream));
        BH_CUDA(m, cudaMemsetAsync(m->d_psi, 0, 8 * nw * sizeof(float), m->stream));
        SrcRecK q;
        q.src_c = sd.src_ir * m->P + sd.src_iz;
        const double V = sd.src_ir == 0
                             ? M_PI * gd.dr * gd.dr * gd.dz
                             : 2.0 * M_PI * (sd.src_ir + 0.5) * gd.dr * gd.dr * gd.dz;
        q.src_scale = (float)(gd.dt / V);
        q.wavelet = wavelet;
        q.recmap = sd.d_recmap;
        q.seis = seis + seis_per_shot * s;
        q.nt = gd.nt;
        q.hist = sd.d_hist;
        const dim3 grd = grid_tiles(gd.nr, sd.nz), blk = block2d();
        if (m->persistent) {
            const int blocks = std::min(n_tiles(gd.nr, sd.nz), m->fwd_blocks);
            BarK b = make_bar(m, blocks);
            BH_CUDA(m, cudaMemsetAsync(m->d_bar, 0, 4 * sizeof(unsigned), m->stream));
            q.n = 0;
            void* args[] = {&g, &C, &S, &q, &b};
            size_t e = prof_begin(m, BH_KERNEL_FWD_PERSIST, 0);
            BH_CUDA(m, cudaLaunchCooperativeKernel((const void*)k_fwd_persist, dim3(blocks), blk,
                                                   args, 0, m->stream));
            prof_end(m, e);
            bh_status st = check_barrier(m);
            if (st != BH_OK) return st;
            continue;
        }
        for (int n = 0; n < gd.nt; ++n) {
            q.n = n;
            size_t e = prof_begin(m, BH_KERNEL_FWD_VEL, n);
            BH_CUDA(m, launch_pdl(k_fwd_vel, grd, blk, m->stream, g, C, S));
            prof_end(m, e);
            e = prof_begin(m, BH_KERNEL_FWD_STRESS, n);
            BH_CUDA(m, launch_pdl(k_fwd_stress, grd, blk, m->stream, g, C, S, q));
            prof_end(m, e);
        }
    }
    m->have_forward = true;
    m->have_gradient = false;
    return BH_OK;
}

bh_status bh_residual_misfit(bh_model* m, const float* seis_mod, const float* seis_obs,
                             float* resid, double* J)
{
    if (!m || !seis_mod || !seis_obs || !resid || !J)
        return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    const size_t n = (size_t)m->nshots * m->nrec_max * m->grid.nt;
    k_misfit<<<1, kRedThreads, 0, m->stream>>>(n, seis_mod, seis_obs, resid, m->d_scal);
    BH_LAUNCH(m);
    BH_CUDA(m, cudaMemcpyAsync(J, m->d_scal, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    BH_CUDA(m, cudaStreamSynchronize(m->stream));
    return BH_OK;
}

bh_status bh_adjoint_gradient(bh_model* m, const float* resid, double* g_lam, double* g_mu,
                              double* g_rho)
{
    if (!m || !resid || !g_lam || !g_mu) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    if (!m->have_forward) return fail(m, BH_ERR_STATE, "bh_forward must come first");
    const bh_grid_desc& gd = m->grid;
    const size_t nw = nrp(m);
    const size_t ng = (size_t)gd.nr * m->nzg;
    const size_t seis_per_shot = (size_t)m->nrec_max * gd.nt;
    BH_CUDA(m, cudaMemsetAsync(g_lam, 0, ng * sizeof(double), m->stream));
    BH_CUDA(m, cudaMemsetAsync(g_mu, 0, ng * sizeof(double), m->stream));
    if (g_rho) BH_CUDA(m, cudaMemsetAsync(g_rho, 0, ng * sizeof(double), m->stream));
    BH_CUDA(m, cudaMemsetAsync(m->d_Hg, 0, 2 * ng * sizeof(double), m->stream));
    FinK f;
    f.g_lam = g_lam;
    f.g_mu = g_mu;
    f.g_rho = g_rho;
    f.H_lam = m->d_Hg;
    f.H_mu = m->d_Hg + ng;
    for (int s = 0; s < m->nshots; ++s) {
        ShotDev& sd = m->shots[s];
        WinK g = make_win(m, sd);
        CoefK C = make_coef(m, sd);
        BH_CUDA(m, cudaMemsetAsync(m->d_state, 0, 6 * nw * sizeof(float), m->stream));
        BH_CUDA(m, cudaMemsetAsync(m->d_psi, 0, 16 * nw * sizeof(float), m->stream));
        BH_CUDA(m, cudaMemsetAsync(m->d_G, 0, 5 * nw * sizeof(float2), m->stream));
        BH_CUDA(m, cudaMemsetAsync(m->d_H, 0, 3 * nw * sizeof(float), m->stream));
        AdjK q;
        q.resid = resid + seis_per_shot * s;
        q.recmap = sd.d_recmap;
        q.nt = gd.nt;
        q.hist = sd.d_hist;
        q.G_lam = m->d_G;
        q.G_munn = m->d_G + nw;
        q.G_murz = m->d_G + 2 * nw;
        q.G_br = m->d_G + 3 * nw;
        q.G_bz = m->d_G + 4 * nw;
        q.H_lam = m->d_H;
        q.H_munn = m->d_H + nw;
        q.H_murz = m->d_H + 2 * nw;
        const dim3 grd = grid2d(gd.nr, sd.nz), blk = block2d();
        const dim3 grt = grid_tiles(gd.nr, sd.nz);
        q.n = gd.nt - 1;
        k_adj_inject<<<(sd.nz + 127) / 128, 128, 0, m->stream>>>(g, make_state(m, 0), q,
                                                                 sd.nrec);
        if (m->persistent) {
            const int blocks = std::min(n_tiles(gd.nr, sd.nz), m->adj_blocks);
            BarK b = make_bar(m, blocks);
            BH_CUDA(m, cudaMemsetAsync(m->d_bar, 0, 4 * sizeof(unsigned), m->stream));
            StateK S0 = make_state(m, 0), S1 = make_state(m, 1);
            void* args[] = {&g, &C, &S0, &S1, &q, &b};
            size_t e = prof_begin(m, BH_KERNEL_ADJ_PERSIST, 0);
            BH_CUDA(m, cudaLaunchCooperativeKernel((const void*)k_adj_persist, dim3(blocks), blk,
                                                   args, 0, m->stream));
            prof_end(m, e);
            bh_status st = check_barrier(m);
            if (st != BH_OK) return st;
            k_finalize<<<grd, blk, 0, m->stream>>>(g, C, q, f);
            BH_LAUNCH(m);
            continue;
        }
        int parity = 0;
        for (int n = gd.nt - 1; n >= 0; --n) {
            q.n = n;
            StateK S = make_state(m, parity);
            size_t e = prof_begin(m, BH_KERNEL_ADJ_STRESS, n);
            BH_CUDA(m, launch_pdl(k_adj_stress, grt, blk, m->stream, g, C, S, q));
            prof_end(m, e);
            e = prof_begin(m, BH_KERNEL_ADJ_VEL, n);
            BH_CUDA(m, launch_pdl(k_adj_vel, grt, blk, m->stream, g, C, S, q));
            prof_end(m, e);
            parity ^= 1;
        }
        k_finalize<<<grd, blk, 0, m->stream>>>(g, C, q, f);
        BH_LAUNCH(m);
    }
    m->have_gradient = true;
    return BH_OK;
}

bh_status bh_get_hessian(bh_model* m, double* H_lam, double* H_mu)
{
    if (!m || !H_lam || !H_mu) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    if (!m->have_gradient) return fail(m, BH_ERR_STATE, "bh_adjoint_gradient must come first");
    const size_t ng = (size_t)m->grid.nr * m->nzg;
    BH_CUDA(m, cudaMemcpyAsync(H_lam, m->d_Hg, ng * sizeof(double), cudaMemcpyDeviceToDevice,
                               m->stream));
    BH_CUDA(m, cudaMemcpyAsync(H_mu, m->d_Hg + ng, ng * sizeof(double),
                               cudaMemcpyDeviceToDevice, m->stream));
    return BH_OK;
}

bh_status bh_precondition(bh_model* m, double* g_lam, double* g_mu, double eps_rel)
{
    if (!m || !g_lam || !g_mu) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    if (!(eps_rel >= 0.0)) return fail(m, BH_ERR_INVALID_ARG, "eps_rel must be >= 0");
    if (!m->have_gradient) return fail(m, BH_ERR_STATE, "bh_adjoint_gradient must come first");
    const size_t ng = (size_t)m->grid.nr * m->nzg;
    k_masked_max2<<<1, kRedThreads, 0, m->stream>>>(ng, m->d_mask, m->d_Hg, m->d_Hg + ng,
                                                    m->d_scal + 2);
    BH_LAUNCH(m);
    k_precondition<<<(unsigned)((ng + 255) / 256), 256, 0, m->stream>>>(
        ng, m->d_mask, m->d_Hg, m->d_Hg + ng, m->d_scal + 2, eps_rel, g_lam, g_mu);
    BH_LAUNCH(m);
    return BH_OK;
}

bh_status bh_update(bh_model* m, const double* g_lam, const double* g_mu, double kappa,
                    double* alpha_out, float* vp_out, float* vs_out)
{
    if (!m || !g_lam || !g_mu) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    if (!(kappa >= 0.0)) return fail(m, BH_ERR_INVALID_ARG, "kappa must be >= 0");
    const size_t ng = (size_t)m->grid.nr * m->nzg;
    k_update_alpha<<<1, kRedThreads, 0, m->stream>>>(ng, m->d_mask, m->d_lam, m->d_mu, g_lam,
                                                     g_mu, kappa, m->d_scal + 4);
    BH_LAUNCH(m);
    const unsigned nb = (unsigned)((ng + 255) / 256);
    k_update_apply<<<nb, 256, 0, m->stream>>>(ng, m->d_mask, g_lam, g_mu, m->d_scal + 4,
                                             m->d_rho, m->d_lam, m->d_mu);
    BH_LAUNCH(m);
    bh_status st = rebuild_coefficients(m);
    if (st != BH_OK) return st;
    if (vp_out || vs_out) {
        k_velocities<<<nb, 256, 0, m->stream>>>(ng, m->d_lam, m->d_mu, m->d_rho, vp_out, vs_out);
        BH_LAUNCH(m);
    }
    if (alpha_out) {
        BH_CUDA(m, cudaMemcpyAsync(alpha_out, m->d_scal + 4, 2 * sizeof(double),
                                   cudaMemcpyDeviceToHost, m->stream));
        BH_CUDA(m, cudaStreamSynchronize(m->stream));
    }
    m->have_forward = m->have_gradient = false;
    return BH_OK;
}

bh_status bh_get_model(bh_model* m, float* vp, float* vs)
{
    if (!m || !vp || !vs) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    const size_t ng = (size_t)m->grid.nr * m->nzg;
    k_velocities<<<(unsigned)((ng + 255) / 256), 256, 0, m->stream>>>(ng, m->d_lam, m->d_mu,
                                                                      m->d_rho, vp, vs);
    BH_LAUNCH(m);
    return BH_OK;
}

bh_status bh_set_option(bh_model* m, const char* key, double value)
{
    if (!m || !key) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    const std::string k(key);
    if (k == "persistent") {
        if (value != 0.0 && (m->fwd_blocks < 1 || m->adj_blocks < 1))
            return fail(m, BH_ERR_UNSUPPORTED, "cooperative launch not available");
        m->persistent = value != 0.0;
    } else if (k == "barrier_timeout_ms") {
        if (!(value > 0.0) || value > 600000.0)
            return fail(m, BH_ERR_INVALID_ARG, "barrier_timeout_ms must be in (0, 600000]");
        m->barrier_timeout_ms = value;
    } else if (k == "barrier_extra_arrivals") {
        if (value < 0.0 || value > 1024.0)
            return fail(m, BH_ERR_INVALID_ARG, "barrier_extra_arrivals must be in [0, 1024]");
        m->barrier_extra = (int)value;
    } else {
        return fail(m, BH_ERR_INVALID_ARG, "unknown option " + k);
    }
    return BH_OK;
}

bh_status bh_profile_enable(bh_model* m, int every)
{
    if (!m || every < 0) return fail(m, BH_ERR_INVALID_ARG, "bad argument");
    m->prof_every = every;
    return BH_OK;
}

bh_status bh_profile_read(bh_model* m, int kernel, double* total_ms, long* launches)
{
    if (!m || !total_ms || !launches || kernel < 0 || kernel >= BH_KERNEL_COUNT)
        return fail(m, BH_ERR_INVALID_ARG, "bad argument");
    if (!m->prof_marks.empty()) {
        BH_CUDA(m, cudaStreamSynchronize(m->stream));
        for (auto& pm : m->prof_marks) {
            float ms = 0.f;
            BH_CUDA(m, cudaEventElapsedTime(&ms, m->ev_pool[pm.second], m->ev_pool[pm.second + 1]));
            m->prof_ms[pm.first] += ms;
            m->prof_n[pm.first] += 1;
        }
        m->prof_marks.clear();
        m->ev_used = 0;
    }
    *total_ms = m->prof_ms[kernel];
    *launches = m->prof_n[kernel];
    return BH_OK;
}

bh_status bh_profile_reset(bh_model* m)
{
    if (!m) return fail(m, BH_ERR_INVALID_ARG, "NULL model");
    double t;
    long n;
    bh_status st = bh_profile_read(m, 0, &t, &n);
    if (st != BH_OK) return st;
    for (int k = 0; k < BH_KERNEL_COUNT; ++k) {
        m->prof_ms[k] = 0.0;
        m->prof_n[k] = 0;
    }
    return BH_OK;
}

}  // extern "C"
