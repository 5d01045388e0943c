// Host runtime and C ABI of libbh (declared in include/bh.h): model object,
// C-PML profiles, shot and tile tables, forward-history window, checkpoint
// schedule, and the drivers that enqueue the kernels of bh_kernels.cuh /
// bh_ops.cuh on the model's stream.
#include "bh.h"
#include "bh_kernels.cuh"
#include "bh_ops.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

using namespace bh;

namespace {

thread_local std::string g_create_error;

// planes (nr x P floats) of one shot's forward and adjoint state
constexpr int kFwdPlanes = 14;  // v_r v_z trr ttt tzz trz + 8 C-PML memories
constexpr int kFields = 6;      // v_r v_z trr ttt tzz trz
constexpr int kAdjPlanes = 35;  // 6 fields + 2 x 8 memories + 5 Kahan pairs + 3 Hessian

struct ShotHost {
    int z0 = 0, nz = 0, src_ir = 0, src_iz = 0, nrec = 0;
    std::vector<int> rec_iz;
    size_t zprof_off = 0, recmap_off = 0;  // offsets into the concatenated tables
};

// One action of the checkpointed reversal (units: segments of L steps).
enum { ACT_ADVANCE = 0, ACT_TAKE = 1, ACT_RESTORE = 2, ACT_REVERSE = 3 };
struct Act {
    int kind, a, b;  // ADVANCE a->b; TAKE slot a <- seg b; RESTORE slot a (seg b); REVERSE seg a
};

}  // namespace

struct bh_model {
    bh_grid_desc grid{};
    int nzg = 0, nshots = 0, nrec_max = 0, P = 0;
    int Pw = 0;                 // row pitch of the shifted coefficient copies
    cudaStream_t stream = nullptr;
    double vpmax = 0.0;
    // model, global [nr][nzg]
    float *d_lam = nullptr, *d_mu = nullptr, *d_rho = nullptr;
    float *d_vp = nullptr, *d_vs = nullptr;  // the model's velocities (as given or as updated)
    float *d_bvr = nullptr, *d_bvz = nullptr, *d_muh = nullptr;
    uint8_t* d_mask = nullptr;
    uint8_t* d_colcov = nullptr;
    // radial profiles: inv_r_int, inv_r_half, ar_int, br_int, ar_half, br_half [6][nr]
    float* d_rprof = nullptr;
    // shots
    std::vector<ShotHost> shots;
    float* d_zprof = nullptr;   // per shot 4 x nz
    int* d_recmap = nullptr;    // per shot nz
    float* d_fwd = nullptr;     // per shot kFwdPlanes planes
    float* d_adj = nullptr;     // per shot kAdjPlanes planes
    float* d_wcoef = nullptr;   // 4 shifted copies x 5 coefficient planes [nr][Pw]
    float* d_fwd2 = nullptr;    // second buffer of the 6 forward fields per shot (fused steps)
    float* d_hist = nullptr;    // per shot (L + 1) x 2 planes
    void* d_snap = nullptr;     // per slot, all shots' kFwdPlanes planes (fp32 or 16-bit)
    float* d_snap_max = nullptr;  // per slot, max |x| of every plane (16-bit snapshots)
    int snap_prec = 0;          // 0 fp32, 1 bf16, 2 fp16
    std::vector<ShotK> h_shots;
    int4* d_tiles = nullptr;    // tiles of every shot group, group after group
    int ntiles = 0;
    int G = 1;                  // shots per launch group (1 .. kGroup)
    std::vector<int> group_tile_off, group_ntiles;  // per group of G shots
    // history window and checkpoint schedule
    int L = 0;                  // steps per history window (nt: store every step)
    int nsnap = 0;              // stored snapshot slots (slot 0 is the zero state)
    int tail = 0;               // last steps whose history the forward sweep stores itself
    int n_tail0 = 0;            // first step of that tail (nt - tail); segments cover [0, n_tail0)
    int hist_slots = 0;         // slots of the history buffer per shot
    std::vector<Act> plan;      // reversal after the forward sweep
    std::vector<std::pair<int, int>> spine;  // (segment, slot) taken during the sweep
    long long recompute_steps = 0;
    long long runs_fwd = 0, runs_adj = 0;  // stepping runs of the last forward / adjoint call
    long long launches = 0;     // kernels this model has launched
    double* d_Hg = nullptr;     // H_lam, H_mu global [2][nr*nzg]
    double* d_scal = nullptr;   // small device scalars
    double* d_part = nullptr;   // per-block partial maxima, 4 x kMaxParts
    bool have_forward = false, have_gradient = false;
    // changes whenever the stored forward history is replaced or invalidated
    // (bh_forward, bh_set_model, bh_update, bh_update_velocity)
    long long state_version = 0;
    std::string err;
    // 1: one cooperative launch per run; 0: one launch per half-step; 2 (auto):
    // cooperative when every block of a shot group has at most one tile
    int persistent = 2;
    int tile_code = 0;          // forward tile code variant (0: one path, 1: per tile class)
    // one launch per half-step and tile class (per-class code only: the
    // adjoint, and the forward with tile code 1)
    // 2: as 1, with the forward's interior tiles in the pipelined kernels;
    // 3: as 1, with one fused launch per forward step for the interior tiles
    int split = 0;
    int pipe_blocks = 0;                  // grid of the pipelined kernels (0: unavailable)
    int pipe_grid = 0;                    // option "pipe_grid": cap on that grid (0: none)
    int tile_order = 0;                   // option "tile_order" (build_tiles)
    TmaMaps maps;                         // tensor maps of the TMA-staged fused step
    bool tma_ok = false;                  // the maps could be encoded ("split" 4)
    int4* d_tiles_cls = nullptr;          // every group's tiles, interior first
    std::vector<int> group_nint;          // interior tiles of each group
    int fwd_blocks = 0, adj_blocks = 0;       // co-resident blocks, 1-shot kernels
    int fwd_blocks_g = 0, adj_blocks_g = 0;   // same, kGroup-shot kernels
    // the adjoint kernels without the density correlation (no g_rho asked)
    int adj_blocks_nr = 0, adj_blocks_g_nr = 0;
    bool adj_rho = true;                      // the running bh_adjoint_gradient wants g_rho
    unsigned* d_bar = nullptr;          // barrier: count, -, error flag
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

// after a kernel launch: count it (bh_get_info "kernel_launches") and check it
#define BH_KERNEL(m)      \
    do {                  \
        ++(m)->launches;  \
        BH_LAUNCH(m);     \
    } while (0)

#define BH_TRY(expr)                   \
    do {                               \
        bh_status s_ = (expr);         \
        if (s_ != BH_OK) return s_;    \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc((void**)p, count * sizeof(T));
}

// Tensor maps of the TMA-staged fused step (k_fwd_step_tma): 3-D views
// (columns, rows, planes) of the two forward field buffers and of the
// coefficient copies, FP32, zero fill out of bounds, no swizzle.  The
// encoder comes from the driver through the runtime's entry-point query.
bool encode_maps(bh_model* m)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    auto one = [&](CUtensorMap* map, void* base, cuuint64_t cols, cuuint64_t rows,
                   cuuint64_t planes, cuuint32_t bx, cuuint32_t by) {
        const cuuint64_t dim[3] = {cols, rows, planes};
        const cuuint64_t stride[2] = {cols * sizeof(float), rows * cols * sizeof(float)};
        const cuuint32_t box[3] = {bx, by, 1};
        const cuuint32_t estride[3] = {1, 1, 1};
        return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dim, stride, box, estride,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    const cuuint64_t nr = m->grid.nr, P = m->P, Pw = m->Pw, ns = m->nshots;
    return one(&m->maps.t[0], m->d_fwd, P, nr, ns * kFwdPlanes, kSZ4, kSR4) &&
           one(&m->maps.t[1], m->d_fwd2, P, nr, ns * kFields, kSZ4, kSR4) &&
           one(&m->maps.v[0], m->d_fwd, P, nr, ns * kFwdPlanes, kSZ, kSR) &&
           one(&m->maps.v[1], m->d_fwd2, P, nr, ns * kFields, kSZ, kSR) &&
           one(&m->maps.w, m->d_wcoef, Pw, nr, 20, kSZ, kSR);
}

void free_model(bh_model* m)
{
    if (!m) return;
    void* bufs[] = {m->d_lam,   m->d_mu,     m->d_rho,   m->d_bvr,    m->d_bvz,    m->d_muh,
                    m->d_vp,    m->d_vs,
                    m->d_mask,  m->d_colcov, m->d_rprof, m->d_zprof,  m->d_recmap, m->d_fwd,
                    m->d_adj,   m->d_hist,   m->d_snap,  m->d_snap_max, m->d_tiles,  m->d_Hg,
                    m->d_scal,  m->d_bar,    m->d_wcoef, m->d_part, m->d_tiles_cls,
                    m->d_fwd2};
    for (void* b : bufs) cudaFree(b);
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

size_t plane(const bh_model* m) { return (size_t)m->grid.nr * m->P; }

dim3 block2d() { return dim3(32, 8); }
// block of the stepping kernels: 8 column groups of 4 nodes x 16 rows
dim3 block_tiles() { return dim3(8, 16); }
dim3 grid2d(int nr, int nz) { return dim3((nz + 31) / 32, (nr + 7) / 8); }

// blocks of the first pass of the masked maxima: about 4 elements per
// thread, at most kMaxParts
int parts_for(size_t n)
{
    const size_t b = (n + 4 * kPartThreads - 1) / (4 * kPartThreads);
    return (int)std::max<size_t>(1, std::min<size_t>(b, kMaxParts));
}

// ------------------------------------------------------ checkpoint schedule
//
// Binomial checkpointing (Griewank and Walther) over segments of L steps:
// with s free snapshot slots and n segments to reverse, let t be the least
// repetition number with C(s + t, s) >= n; advancing to the split
// m = l + max(1, n - C(s - 1 + t, s - 1)) and reversing [m, r) with s - 1
// slots and [l, m) with s slots keeps every segment within t advances.

double binom(int s, int t)
{
    double b = 1.0;
    for (int k = 1; k <= s; ++k) b = b * (t + k) / k;  // C(s + t, s)
    return b;
}

void rev(int l, int r, int slot_l, int s, int next_slot, std::vector<Act>& out)
{
    const int n = r - l;
    if (n <= 0) return;
    if (n == 1) {
        out.push_back({ACT_RESTORE, slot_l, l});
        out.push_back({ACT_REVERSE, l, 0});
        return;
    }
    if (s == 0) {
        for (int k = r - 1; k >= l; --k) {
            out.push_back({ACT_RESTORE, slot_l, l});
            if (k > l) out.push_back({ACT_ADVANCE, l, k});
            out.push_back({ACT_REVERSE, k, 0});
        }
        return;
    }
    int t = 1;
    while (binom(s, t) < n) ++t;
    int mp = n - (int)std::min<double>(binom(s - 1, t), (double)n);
    mp = std::max(1, std::min(mp, n - 1));
    const int m = l + mp;
    out.push_back({ACT_RESTORE, slot_l, l});
    out.push_back({ACT_ADVANCE, l, m});
    out.push_back({ACT_TAKE, next_slot, m});
    rev(m, r, next_slot, s - 1, next_slot + 1, out);
    rev(l, m, slot_l, s, next_slot, out);
}

// Full action list for nseg segments with nsnap stored slots; the leading
// RESTORE / ADVANCE / TAKE chain that walks forward from segment 0 is moved
// into the forward sweep (its snapshots are taken on the way).
void build_plan(int nseg, int nsnap, std::vector<Act>* plan,
                std::vector<std::pair<int, int>>* spine, long long* adv_segments)
{
    std::vector<Act> all;
    rev(0, nseg, 0, nsnap, 1, all);
    size_t k = 0;
    int pos = 0, pos_slot = 0;
    spine->clear();
    while (k + 2 < all.size() && all[k].kind == ACT_RESTORE && all[k].a == pos_slot &&
           all[k + 1].kind == ACT_ADVANCE && all[k + 1].a == pos && all[k + 2].kind == ACT_TAKE) {
        pos = all[k + 2].b;
        pos_slot = all[k + 2].a;
        spine->push_back({pos, pos_slot});
        k += 3;
    }
    plan->assign(all.begin() + k, all.end());
    long long adv = 0;
    for (const Act& a : *plan)
        if (a.kind == ACT_ADVANCE) adv += a.b - a.a;
    *adv_segments = adv;
}

// ------------------------------------------------------------ model setup

bh_status rebuild_coefficients(bh_model* m)
{
    const int nr = m->grid.nr, nzg = m->nzg;
    k_setup_nodes<<<grid2d(nr, nzg), block2d(), 0, m->stream>>>(nr, nzg, m->d_mu, m->d_rho,
                                                                m->d_bvr, m->d_bvz, m->d_muh);
    BH_KERNEL(m);
    dim3 gw = grid2d(nr, m->Pw);
    gw.z = 4;
    k_shift_coefs<<<gw, block2d(), 0, m->stream>>>(nr, nzg, m->Pw, m->d_lam, m->d_mu, m->d_muh,
                                                   m->d_bvr, m->d_bvz, m->d_wcoef);
    BH_KERNEL(m);
    return BH_OK;
}

bh_status load_model(bh_model* m, const float* vp, const float* vs, const float* rho,
                     bool first)
{
    const int nr = m->grid.nr, nzg = m->nzg;
    const size_t n = (size_t)nr * nzg;
    // CFL check and C-PML d0 need max Vp
    k_max_f32<<<1, kRedThreads, 0, m->stream>>>(n, vp, m->d_scal);
    BH_KERNEL(m);
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
    k_setup_cells<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, m->stream>>>(
        (int)n, vp, vs, rho, m->d_lam, m->d_mu, m->d_rho, m->d_vp, m->d_vs);
    BH_KERNEL(m);
    if (first) {
        k_setup_mask<<<grid2d(nr, nzg), block2d(), 0, m->stream>>>(nr, nzg, g.npml_r, vs,
                                                                   m->d_colcov, m->d_mask);
        BH_KERNEL(m);
    }
    BH_TRY(rebuild_coefficients(m));
    m->have_forward = m->have_gradient = false;
    ++m->state_version;
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
    const double Lz = g.npml_z * g.dz;
    const double d0z = g.npml_z > 0 ? -3.0 * m->vpmax * std::log(R) / (2.0 * Lz) : 0.0;
    std::vector<float> zp;
    std::vector<int> recmap;
    for (auto& s : m->shots) {
        const int nz = s.nz, P = m->P;
        s.zprof_off = zp.size();
        s.recmap_off = recmap.size();
        // 4 profiles of P entries each (zero beyond nz: read as float4 rows)
        zp.resize(zp.size() + 4 * (size_t)P, 0.f);
        float* z = zp.data() + s.zprof_off;
        for (int j = 0; j < nz; ++j)
            for (int h = 0; h < 2; ++h) {
                double zz = (j + 0.5 * h) * g.dz, x = 0.0;
                if (g.npml_z > 0) {
                    double xt = ((g.npml_z - 0.5) * g.dz - zz) / Lz;
                    double xb = (zz - (nz - g.npml_z - 0.5) * g.dz) / Lz;
                    x = std::max(xt, xb);
                }
                double a, b;
                pml_ab(x, d0z, alpha_max, g.dt, &a, &b);
                z[(2 * h) * P + j] = (float)a;
                z[(2 * h + 1) * P + j] = (float)b;
            }
        recmap.resize(recmap.size() + nz, -1);
        for (int k = 0; k < s.nrec; ++k) recmap[s.recmap_off + s.rec_iz[k]] = k;
    }
    BH_CUDA(m, dalloc(&m->d_zprof, zp.size()));
    BH_CUDA(m, dalloc(&m->d_recmap, recmap.size()));
    BH_CUDA(m, cudaMemcpyAsync(m->d_rprof, rp.data(), rp.size() * sizeof(float),
                               cudaMemcpyHostToDevice, m->stream));
    BH_CUDA(m, cudaMemcpyAsync(m->d_zprof, zp.data(), zp.size() * sizeof(float),
                               cudaMemcpyHostToDevice, m->stream));
    BH_CUDA(m, cudaMemcpyAsync(m->d_recmap, recmap.data(), recmap.size() * sizeof(int),
                               cudaMemcpyHostToDevice, m->stream));
    // host vectors must outlive the copies
    BH_CUDA(m, cudaStreamSynchronize(m->stream));
    return BH_OK;
}

bh_status build_tiles(bh_model* m);

// Per-shot descriptors (pointers into the arenas) and the tile table.
bh_status setup_shots(bh_model* m)
{
    const bh_grid_desc& gd = m->grid;
    const int nr = gd.nr;
    const size_t pl = plane(m);
    m->h_shots.resize(m->nshots);
    for (int s = 0; s < m->nshots; ++s) {
        const ShotHost& sh = m->shots[s];
        ShotK& k = m->h_shots[s];
        memset(&k, 0, sizeof(k));
        k.g.nr = nr;
        k.g.nz = sh.nz;
        k.g.P = m->P;
        k.g.Pw = m->Pw;
        k.g.nzg = m->nzg;
        k.g.z0 = sh.z0;
        k.g.npml_r = gd.npml_r;
        k.g.npml_z = gd.npml_z;
        k.g.dt = (float)gd.dt;
        k.g.inv_dr = (float)(1.0 / gd.dr);
        k.g.inv_dz = (float)(1.0 / gd.dz);
        CoefK& C = k.C;
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
        const float* zp = m->d_zprof + sh.zprof_off;
        C.az_int = zp;
        C.bz_int = zp + m->P;
        C.az_half = zp + 2 * m->P;
        C.bz_half = zp + 3 * m->P;
        // the shifted copy in which the window's column 0 is 16-byte aligned
        const int kc = (4 - (sh.z0 & 3)) & 3;
        const size_t plw = (size_t)nr * m->Pw;
        const float* wc = m->d_wcoef + (size_t)kc * 5 * plw + sh.z0 + kc;
        C.w_lam = wc;
        C.w_mu = wc + plw;
        C.w_muh = wc + 2 * plw;
        C.w_bvr = wc + 3 * plw;
        C.w_bvz = wc + 4 * plw;
        float* f = m->d_fwd + (size_t)s * kFwdPlanes * pl;
        k.swap = (long long)((m->d_fwd2 + (size_t)s * kFields * pl) - f);
        float* a = m->d_adj + (size_t)s * kAdjPlanes * pl;
        StateK* views[3] = {&k.Sf, &k.Sa[0], &k.Sa[1]};
        for (int v = 0; v < 3; ++v) {
            float* b = v == 0 ? f : a;
            StateK& S = *views[v];
            S.vr = b;
            S.vz = b + pl;
            S.trr = b + 2 * pl;
            S.ttt = b + 3 * pl;
            S.tzz = b + 4 * pl;
            S.trz = b + 5 * pl;
            for (int q = 0; q < 8; ++q) {
                float* bank_a = b + (6 + q) * pl;
                float* bank_b = a + (14 + q) * pl;
                if (v == 0) S.psi[q] = S.psi_w[q] = bank_a;
                else if (v == 1) { S.psi[q] = bank_a; S.psi_w[q] = bank_b; }
                else { S.psi[q] = bank_b; S.psi_w[q] = bank_a; }
            }
        }
        k.q.src_c = sh.src_ir * m->P + sh.src_iz;
        const double V = sh.src_ir == 0 ? M_PI * gd.dr * gd.dr * gd.dz
                                        : 2.0 * M_PI * (sh.src_ir + 0.5) * gd.dr * gd.dr * gd.dz;
        k.q.src_scale = (float)(gd.dt / V);
        k.q.recmap = m->d_recmap + sh.recmap_off;
        k.q.nt = gd.nt;
        k.a.recmap = k.q.recmap;
        k.a.nt = gd.nt;
        k.a.G_lam = (float2*)(a + 22 * pl);
        k.a.G_munn = (float2*)(a + 24 * pl);
        k.a.G_murz = (float2*)(a + 26 * pl);
        k.a.G_br = (float2*)(a + 28 * pl);
        k.a.G_bz = (float2*)(a + 30 * pl);
        k.a.H_lam = a + 32 * pl;
        k.a.H_munn = a + 33 * pl;
        k.a.H_murz = a + 34 * pl;
        k.hist = m->d_hist + (size_t)s * m->hist_slots * 2 * pl;
    }
    return build_tiles(m);
}

// Tile table of every shot group of G shots, group after group.  Within a
// group the tiles are ordered (option "tile_order") 0: by global column,
// then row, then shot: tiles of several shots at one place of the model run
// together and share the coefficient copies' lines in L2; 1: by shot, then
// row, then column: the blocks resident at one time cover long runs of
// each row (DRAM pages read whole).  The order changes no result.
bh_status build_tiles(bh_model* m)
{
    const bh_grid_desc& gd = m->grid;
    const int nr = gd.nr, G = m->G;
    std::vector<int4> tiles;
    m->group_tile_off.clear();
    m->group_ntiles.clear();
    for (int s = 0; s < m->nshots; ++s) {
        const ShotHost& sh = m->shots[s];
        if (s % G == 0) {
            m->group_tile_off.push_back((int)tiles.size());
            m->group_ntiles.push_back(0);
        }
        for (int i0 = 0; i0 < nr; i0 += kTR)
            for (int j0 = 0; j0 < sh.nz; j0 += kTZ) {
                // a tile reads nodes i0-2 .. i0+17, j0-4 .. j0+35; a layer
                // coefficient is non-zero from row nr - npml_r and in the
                // first / last npml_z columns (one node of margin each way)
                const bool radial = gd.npml_r > 0 && i0 + kTR + kH >= nr - gd.npml_r - 1;
                const bool axial = gd.npml_z > 0 &&
                                   (j0 - 4 <= gd.npml_z + 1 || j0 + kTZ + 4 >= sh.nz - gd.npml_z - 2);
                const bool last = j0 - 4 <= sh.nz - 1 && sh.nz - 1 <= j0 + kTZ + 3;
                tiles.push_back(make_int4(s % G, i0, j0,
                                          ((radial || axial) ? TILE_PML : 0) |
                                              (last ? TILE_LAST : 0)));
                m->group_ntiles.back()++;
            }
        if (m->tile_order == 0 && (s % G == G - 1 || s == m->nshots - 1)) {
            const int g0 = m->group_tile_off.back();
            const int sbase = s - s % G;
            std::stable_sort(tiles.begin() + g0, tiles.end(), [&](const int4& a, const int4& b) {
                const int za = m->shots[sbase + a.x].z0 + a.z, zb = m->shots[sbase + b.x].z0 + b.z;
                if (za != zb) return za < zb;
                if (a.y != b.y) return a.y < b.y;
                return a.x < b.x;
            });
        }
    }
    m->ntiles = (int)tiles.size();
    // the same tables with every group's interior tiles first, for launches
    // of one tile class
    std::vector<int4> cls(tiles);
    m->group_nint.clear();
    for (size_t grp = 0; grp < m->group_tile_off.size(); ++grp) {
        auto b = cls.begin() + m->group_tile_off[grp];
        auto mid = std::stable_partition(b, b + m->group_ntiles[grp],
                                         [](const int4& t) { return !(t.w & TILE_PML); });
        m->group_nint.push_back((int)(mid - b));
    }
    cudaFree(m->d_tiles);
    cudaFree(m->d_tiles_cls);
    m->d_tiles = m->d_tiles_cls = nullptr;
    BH_CUDA(m, dalloc(&m->d_tiles, tiles.size()));
    BH_CUDA(m, dalloc(&m->d_tiles_cls, cls.size()));
    BH_CUDA(m, cudaMemcpyAsync(m->d_tiles, tiles.data(), tiles.size() * sizeof(int4),
                               cudaMemcpyHostToDevice, m->stream));
    BH_CUDA(m, cudaMemcpyAsync(m->d_tiles_cls, cls.data(), cls.size() * sizeof(int4),
                               cudaMemcpyHostToDevice, m->stream));
    BH_CUDA(m, cudaStreamSynchronize(m->stream));
    return BH_OK;
}

// shot table of one group, passed by value to the stepping kernels
template <int N>
ShotTable<N> group_table(const bh_model* m, int grp)
{
    ShotTable<N> T;
    memset(&T, 0, sizeof(T));
    for (int k = 0; k < N && k < m->G && grp * m->G + k < m->nshots; ++k)
        T.s[k] = m->h_shots[grp * m->G + k];
    return T;
}

// ------------------------------------------------------------------ runs

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

BarK make_bar(const bh_model* m, int blocks)
{
    BarK b;
    b.count = m->d_bar;
    b.err = (int*)(m->d_bar + 2);
    b.expected = (unsigned)blocks + (unsigned)m->barrier_extra;
    b.timeout_ns = (unsigned long long)(m->barrier_timeout_ms * 1e6);
    return b;
}

// Launch form of one shot group.  The persistent kernels overlap a block's
// barrier wait with its own-node work but run a block's tiles one after the
// other; when a group has more tiles than co-resident blocks, one launch per
// half-step lets the block scheduler overlap one block's staging with
// another's compute and wins (GB300: 16 % at 3125 tiles, 44 % at 795 tiles;
// the persistent form wins by 4.5 % at 750 tiles).
int adj_blocks_for(const bh_model* m, bool one_shot)
{
    if (m->adj_rho) return one_shot ? m->adj_blocks : m->adj_blocks_g;
    return one_shot ? m->adj_blocks_nr : m->adj_blocks_g_nr;
}

bool persistent_for(const bh_model* m, int grp, bool adjoint)
{
    if (m->persistent != 2) return m->persistent != 0;
    const bool one = m->G == 1;
    const int blocks = adjoint ? adj_blocks_for(m, one) : (one ? m->fwd_blocks : m->fwd_blocks_g);
    return m->group_ntiles[grp] <= blocks;
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

// the interior and C-PML runs of a group for launches of one tile class
void class_runs(const bh_model* m, int grp, const RunK& r, RunK* ri, RunK* rp)
{
    *ri = r;
    *rp = r;
    ri->tiles = m->d_tiles_cls + m->group_tile_off[grp];
    ri->ntiles = m->group_nint[grp];
    rp->tiles = ri->tiles + ri->ntiles;
    rp->ntiles = r.ntiles - ri->ntiles;
}

RunK make_run(const bh_model* m, int grp, int n0, int n1, int hist_n0, bool record)
{
    RunK r;
    r.tiles = m->d_tiles + m->group_tile_off[grp];
    r.ntiles = m->group_ntiles[grp];
    r.n0 = n0;
    r.n1 = n1;
    r.hist_n0 = hist_n0;
    r.record = record ? 1 : 0;
    r.nt = m->grid.nt;
    return r;
}

// Forward steps n0 .. n1-1 of the shots of one group, tile code variant V.
template <int N, int V>
bh_status run_forward_group(bh_model* m, int grp, int n0, int n1, int hist_n0, bool record)
{
    RunK r = make_run(m, grp, n0, n1, hist_n0, record);
    ShotTable<N> T = group_table<N>(m, grp);
    const dim3 blk = block_tiles();
    if (persistent_for(m, grp, false)) {
        const int blocks = std::min(r.ntiles, N == 1 ? m->fwd_blocks : m->fwd_blocks_g);
        BarK b = make_bar(m, blocks);
        BH_CUDA(m, cudaMemsetAsync(m->d_bar, 0, 4 * sizeof(unsigned), m->stream));
        void* args[] = {&r, &b, &T};
        size_t e = prof_begin(m, BH_KERNEL_FWD_PERSIST, 0);
        BH_CUDA(m, cudaLaunchCooperativeKernel((const void*)k_fwd_persist<N, V>, dim3(blocks), blk,
                                               args, 0, m->stream));
        ++m->launches;
        prof_end(m, e);
        return check_barrier(m);
    }
    const dim3 grd(r.ntiles);
    if (V == 1 && (m->split == 3 || (m->split == 4 && m->tma_ok))) {
        // fused steps: the fields ping-pong between the two buffers and end
        // in buffer 0 (snapshots and the next run start there)
        RunK ri, rp;
        class_runs(m, grp, r, &ri, &rp);
        for (int n = n0; n < n1; ++n) {
            const int pp = (n - n0) & 1;
            size_t e = prof_begin(m, BH_KERNEL_FWD_STEP, n);
            if (ri.ntiles && m->split == 4) {
                BH_CUDA(m, launch_pdl(k_fwd_step_tma<N>, dim3(ri.ntiles), blk, m->stream, ri, n,
                                      pp, grp * m->G, (int*)(m->d_bar + 2), m->maps, T));
                ++m->launches;
            } else if (ri.ntiles) {
                BH_CUDA(m, launch_pdl(k_fwd_step<N>, dim3(ri.ntiles), blk, m->stream, ri, n, pp, T));
                ++m->launches;
            }
            if (rp.ntiles) {
                BH_CUDA(m, launch_pdl(k_fwd_vel_c<N, PM_PML>, dim3(rp.ntiles), blk, m->stream, rp,
                                      n, pp, T));
                BH_CUDA(m, launch_pdl(k_fwd_stress_c<N, PM_PML>, dim3(rp.ntiles), blk, m->stream,
                                      rp, n, pp, T));
                m->launches += 2;
            }
            prof_end(m, e);
        }
        if ((n1 - n0) & 1) {
            const size_t pl = plane(m);
            const int s0 = grp * m->G, ns = std::min(m->G, m->nshots - s0);
            BH_CUDA(m, cudaMemcpy2DAsync(m->d_fwd + (size_t)s0 * kFwdPlanes * pl,
                                         kFwdPlanes * pl * sizeof(float),
                                         m->d_fwd2 + (size_t)s0 * kFields * pl,
                                         kFields * pl * sizeof(float), kFields * pl * sizeof(float),
                                         ns, cudaMemcpyDeviceToDevice, m->stream));
        }
        return BH_OK;
    }
    if (V == 1 && m->split) {
        RunK ri, rp;
        class_runs(m, grp, r, &ri, &rp);
        const bool pipe = m->split == 2 && m->pipe_blocks > 0;
        const int pg = m->pipe_grid > 0 ? std::min(m->pipe_grid, m->pipe_blocks) : m->pipe_blocks;
        for (int n = n0; n < n1; ++n) {
            size_t e = prof_begin(m, BH_KERNEL_FWD_VEL, n);
            if (ri.ntiles && pipe) {
                BH_CUDA(m, launch_pdl(k_fwd_vel_pipe<N>, dim3(std::min(ri.ntiles, pg)), blk,
                                      m->stream, ri, n, T));
                ++m->launches;
            } else if (ri.ntiles) {
                BH_CUDA(m, launch_pdl(k_fwd_vel_c<N, PM_INTERIOR>, dim3(ri.ntiles), blk,
                                      m->stream, ri, n, -1, T));
                ++m->launches;
            }
            if (rp.ntiles) {
                BH_CUDA(m, launch_pdl(k_fwd_vel_c<N, PM_PML>, dim3(rp.ntiles), blk, m->stream,
                                      rp, n, -1, T));
                ++m->launches;
            }
            prof_end(m, e);
            e = prof_begin(m, BH_KERNEL_FWD_STRESS, n);
            if (ri.ntiles && pipe) {
                BH_CUDA(m, launch_pdl(k_fwd_stress_pipe<N>,
                                      dim3(std::min(ri.ntiles, pg)), blk, m->stream, ri, n, T));
                ++m->launches;
            } else if (ri.ntiles) {
                BH_CUDA(m, launch_pdl(k_fwd_stress_c<N, PM_INTERIOR>, dim3(ri.ntiles), blk,
                                      m->stream, ri, n, -1, T));
                ++m->launches;
            }
            if (rp.ntiles) {
                BH_CUDA(m, launch_pdl(k_fwd_stress_c<N, PM_PML>, dim3(rp.ntiles), blk,
                                      m->stream, rp, n, -1, T));
                ++m->launches;
            }
            prof_end(m, e);
        }
        return BH_OK;
    }
    for (int n = n0; n < n1; ++n) {
        size_t e = prof_begin(m, BH_KERNEL_FWD_VEL, n);
        BH_CUDA(m, launch_pdl(k_fwd_vel<N, V>, grd, blk, m->stream, r, n, T));
        ++m->launches;
        prof_end(m, e);
        e = prof_begin(m, BH_KERNEL_FWD_STRESS, n);
        BH_CUDA(m, launch_pdl(k_fwd_stress<N, V>, grd, blk, m->stream, r, n, T));
        ++m->launches;
        prof_end(m, e);
    }
    return BH_OK;
}

// Reverse steps n1-1 down to n0 of the shots of one group; RHO: with the
// density correlation.
template <int N, bool RHO>
bh_status run_adjoint_group(bh_model* m, int grp, int n0, int n1, int hist_n0)
{
    RunK r = make_run(m, grp, n0, n1, hist_n0, false);
    ShotTable<N> T = group_table<N>(m, grp);
    const dim3 blk = block_tiles();
    if (persistent_for(m, grp, true)) {
        const int blocks = std::min(r.ntiles, adj_blocks_for(m, N == 1));
        BarK b = make_bar(m, blocks);
        BH_CUDA(m, cudaMemsetAsync(m->d_bar, 0, 4 * sizeof(unsigned), m->stream));
        void* args[] = {&r, &b, &T};
        size_t e = prof_begin(m, BH_KERNEL_ADJ_PERSIST, 0);
        BH_CUDA(m, cudaLaunchCooperativeKernel((const void*)k_adj_persist<N, RHO>, dim3(blocks),
                                               blk, args, 0, m->stream));
        ++m->launches;
        prof_end(m, e);
        return check_barrier(m);
    }
    const dim3 grd(r.ntiles);
    if (m->split) {
        RunK ri, rp;
        class_runs(m, grp, r, &ri, &rp);
        for (int n = n1 - 1; n >= n0; --n) {
            size_t e = prof_begin(m, BH_KERNEL_ADJ_STRESS, n);
            if (ri.ntiles) {
                BH_CUDA(m, launch_pdl(k_adj_stress_c<N, RHO, PM_INTERIOR>, dim3(ri.ntiles), blk,
                                      m->stream, ri, n, T));
                ++m->launches;
            }
            if (rp.ntiles) {
                BH_CUDA(m, launch_pdl(k_adj_stress_c<N, RHO, PM_PML>, dim3(rp.ntiles), blk,
                                      m->stream, rp, n, T));
                ++m->launches;
            }
            prof_end(m, e);
            e = prof_begin(m, BH_KERNEL_ADJ_VEL, n);
            if (ri.ntiles) {
                BH_CUDA(m, launch_pdl(k_adj_vel_c<N, RHO, PM_INTERIOR>, dim3(ri.ntiles), blk,
                                      m->stream, ri, n, T));
                ++m->launches;
            }
            if (rp.ntiles) {
                BH_CUDA(m, launch_pdl(k_adj_vel_c<N, RHO, PM_PML>, dim3(rp.ntiles), blk,
                                      m->stream, rp, n, T));
                ++m->launches;
            }
            prof_end(m, e);
        }
        return BH_OK;
    }
    for (int n = n1 - 1; n >= n0; --n) {
        size_t e = prof_begin(m, BH_KERNEL_ADJ_STRESS, n);
        BH_CUDA(m, launch_pdl(k_adj_stress<N, RHO>, grd, blk, m->stream, r, n, T));
        ++m->launches;
        prof_end(m, e);
        e = prof_begin(m, BH_KERNEL_ADJ_VEL, n);
        BH_CUDA(m, launch_pdl(k_adj_vel<N, RHO>, grd, blk, m->stream, r, n, T));
        ++m->launches;
        prof_end(m, e);
    }
    return BH_OK;
}

// launches per half-step of a group split by tile class
int class_launches(const bh_model* m, int grp)
{
    return (m->group_nint[grp] > 0) + (m->group_ntiles[grp] - m->group_nint[grp] > 0);
}

// Forward steps n0 .. n1-1 of every shot, group by group.
bh_status run_forward(bh_model* m, int n0, int n1, int hist_n0, bool record, long long* runs)
{
    if (n1 <= n0) return BH_OK;
    const int ngroups = (int)m->group_ntiles.size();
    const bool tma = m->split == 4 && m->tile_code == 1 && m->tma_ok;
    if (tma) BH_CUDA(m, cudaMemsetAsync(m->d_bar + 2, 0, sizeof(unsigned), m->stream));
    for (int grp = 0; grp < ngroups; ++grp) {
        const int nint = m->group_nint[grp], npml = m->group_ntiles[grp] - nint;
        *runs += persistent_for(m, grp, false) ? 1
                 : (m->split >= 3 && m->tile_code == 1)
                     ? (long long)(n1 - n0) * ((nint > 0) + 2 * (npml > 0))
                     : 2 * (n1 - n0) * ((m->split && m->tile_code == 1) ? class_launches(m, grp) : 1);
        const bool one = m->G == 1;
        if (m->tile_code == 0) {
            if (one) BH_TRY((run_forward_group<1, 0>(m, grp, n0, n1, hist_n0, record)));
            else BH_TRY((run_forward_group<kGroup, 0>(m, grp, n0, n1, hist_n0, record)));
        } else {
            if (one) BH_TRY((run_forward_group<1, 1>(m, grp, n0, n1, hist_n0, record)));
            else BH_TRY((run_forward_group<kGroup, 1>(m, grp, n0, n1, hist_n0, record)));
        }
    }
    if (tma) {
        // a TMA copy that never completed left its flag (bounded wait)
        int err = 0;
        BH_CUDA(m, cudaMemcpyAsync(&err, m->d_bar + 2, sizeof(int), cudaMemcpyDeviceToHost,
                                   m->stream));
        BH_CUDA(m, cudaStreamSynchronize(m->stream));
        if (err)
            return fail(m, BH_ERR_TIMEOUT,
                        "a tensor copy of the fused forward step did not complete; results are "
                        "invalid");
    }
    return BH_OK;
}

// Reverse steps n1-1 down to n0 of every shot; the history window starts at hist_n0.
bh_status run_adjoint(bh_model* m, int n0, int n1, int hist_n0, long long* runs)
{
    if (n1 <= n0) return BH_OK;
    const int ngroups = (int)m->group_ntiles.size();
    for (int grp = 0; grp < ngroups; ++grp) {
        *runs += persistent_for(m, grp, true)
                     ? 1
                     : 2 * (n1 - n0) * (m->split ? class_launches(m, grp) : 1);
        const bool one = m->G == 1;
        if (m->adj_rho) {
            if (one) BH_TRY((run_adjoint_group<1, true>(m, grp, n0, n1, hist_n0)));
            else BH_TRY((run_adjoint_group<kGroup, true>(m, grp, n0, n1, hist_n0)));
        } else {
            if (one) BH_TRY((run_adjoint_group<1, false>(m, grp, n0, n1, hist_n0)));
            else BH_TRY((run_adjoint_group<kGroup, false>(m, grp, n0, n1, hist_n0)));
        }
    }
    return BH_OK;
}

// forward state of every shot <-> snapshot slot (slot 0 is the zero state)
bh_status snapshot(bh_model* m, int slot, bool take)
{
    const size_t pl = plane(m);
    const size_t bytes = kFwdPlanes * pl * sizeof(float);
    if (slot == 0) {
        if (take) return fail(m, BH_ERR_STATE, "snapshot slot 0 is the initial state");
        BH_CUDA(m, cudaMemsetAsync(m->d_fwd, 0, bytes * m->nshots, m->stream));
        return BH_OK;
    }
    const size_t per_slot = (size_t)m->nshots * kFwdPlanes * pl;
    if (m->snap_prec == 0) {
        float* snap = (float*)m->d_snap + (size_t)(slot - 1) * per_slot;
        if (take)
            BH_CUDA(m, cudaMemcpyAsync(snap, m->d_fwd, bytes * m->nshots,
                                       cudaMemcpyDeviceToDevice, m->stream));
        else
            BH_CUDA(m, cudaMemcpyAsync(m->d_fwd, snap, bytes * m->nshots,
                                       cudaMemcpyDeviceToDevice, m->stream));
        return BH_OK;
    }
    // 16-bit snapshot with a power-of-two scale per plane
    uint16_t* snap = (uint16_t*)m->d_snap + (size_t)(slot - 1) * per_slot;
    float* mx = m->d_snap_max + (size_t)(slot - 1) * m->nshots * kFwdPlanes;
    const unsigned nb = (unsigned)std::min<size_t>((per_slot + 255) / 256, 152 * 16);
    if (take) {
        k_plane_maxabs<<<m->nshots * kFwdPlanes, 256, 0, m->stream>>>(m->d_fwd, pl, mx);
        BH_KERNEL(m);
        k_snap_encode<<<nb, 256, 0, m->stream>>>(m->d_fwd, pl, per_slot, mx, m->snap_prec, snap);
    } else {
        k_snap_decode<<<nb, 256, 0, m->stream>>>(snap, pl, per_slot, mx, m->snap_prec, m->d_fwd);
    }
    BH_KERNEL(m);
    return BH_OK;
}

// History plan under a byte cap.  The nt steps are split into segments of L
// steps over [0, n_tail0) and a tail [n_tail0, nt) whose history the forward
// sweep stores as it goes (tail = nt: every step stored, nothing re-run).
// Each segment is re-run once into the history window before its adjoint,
// from a snapshot taken during the sweep (binomial schedule when there are
// fewer snapshots than segments).  Memory: (max(tail, L) + 1) history slots
// plus the snapshots.  Recomputed steps: the segments' steps plus the
// schedule's advances.  Among the plans that fit, the fewest recomputed
// steps win, then the least memory.
struct HistPlan {
    int L = 0, nsnap = 0, tail = 0;
    long long recompute = -1;
    double bytes = 0.0;
};

HistPlan choose_history_plan(int nt, double hist_step, double snap, double cap)
{
    HistPlan best;
    auto consider = [&](int L, int s, int tail, long long cost, double bytes) {
        if (bytes > cap) return;
        if (best.recompute < 0 || cost < best.recompute ||
            (cost == best.recompute && bytes < best.bytes)) {
            best.L = L;
            best.nsnap = s;
            best.tail = tail;
            best.recompute = cost;
            best.bytes = bytes;
        }
    };
    // every step stored
    consider(nt, 0, nt, 0, (nt + 1.0) * hist_step);
    if (best.recompute == 0) return best;
    // a stored tail and a snapshot at every earlier segment start: nseg' =
    // segments before the tail, recompute = nseg' L (no advances)
    for (int L = 1; L < nt; ++L) {
        const int nseg = (nt + L - 1) / L;
        for (int nsp = 1; nsp < nseg; ++nsp) {
            const int n0 = nsp * L;
            const int tail = nt - n0;
            const double bytes = (std::max(tail, L) + 1.0) * hist_step + (nsp - 1.0) * snap;
            if (bytes <= cap) {
                // more segments only cost more recompute: the first that fits
                consider(L, nsp - 1, tail, n0, bytes);
                break;
            }
            // with L hist_step > snap every further segment frees memory;
            // otherwise nothing later fits either
            if (L * hist_step <= snap) break;
        }
    }
    if (best.recompute >= 0) return best;
    // no room for a snapshot at every segment: no tail, the window plus the
    // snapshots that fit, binomial schedule
    std::vector<int> Ls;
    for (int L = 1; L < nt; L *= 2) Ls.push_back(L);
    for (int L : {3, 5, 6, 10, 12, 20, 24, 40, 48, 80, 96, 100, 160, 200, 250, 400, 500})
        if (L < nt) Ls.push_back(L);
    for (int L : Ls) {
        const double hist = (L + 1.0) * hist_step;
        if (hist > cap) continue;
        const int nseg = (nt + L - 1) / L;
        long long s = (long long)((cap - hist) / snap);
        s = std::min<long long>(s, nseg - 1);
        if (s < 0) continue;
        if (nseg > 2000 && s == 0) continue;  // quadratic plans are not worth listing
        std::vector<Act> plan;
        std::vector<std::pair<int, int>> spine;
        long long adv = 0;
        build_plan(nseg, (int)s, &plan, &spine, &adv);
        consider(L, (int)s, 0, adv * (long long)L + nt, hist + s * snap);
    }
    return best;
}

bh_status plan_checkpoints(bh_model* m, size_t cap)
{
    const int nt = m->grid.nt;
    const double pl_bytes = (double)plane(m) * sizeof(float) * m->nshots;
    const double snap_bytes = kFwdPlanes * pl_bytes * (m->snap_prec ? 0.5 : 1.0);
    const HistPlan hp = choose_history_plan(nt, 2.0 * pl_bytes, snap_bytes, (double)cap);
    if (hp.recompute < 0)
        return fail(m, BH_ERR_OOM, "checkpoint_cap_bytes too small for one history window");
    m->L = hp.L;
    m->nsnap = hp.nsnap;
    m->tail = hp.tail;
    m->n_tail0 = nt - hp.tail;
    m->hist_slots = (hp.tail >= nt ? nt : std::max(hp.tail, hp.L)) + 1;
    m->plan.clear();
    m->spine.clear();
    long long adv = 0;
    if (m->n_tail0 > 0)
        build_plan((m->n_tail0 + hp.L - 1) / hp.L, hp.nsnap, &m->plan, &m->spine, &adv);
    m->recompute_steps = adv * hp.L + m->n_tail0;
    return BH_OK;
}

// the model's velocities / density into caller buffers (each may be NULL)
bh_status copy_model_out(bh_model* m, float* vp, float* vs, float* rho)
{
    const size_t bytes = (size_t)m->grid.nr * m->nzg * sizeof(float);
    const float* src[3] = {m->d_vp, m->d_vs, m->d_rho};
    float* dst[3] = {vp, vs, rho};
    for (int q = 0; q < 3; ++q)
        if (dst[q])
            BH_CUDA(m, cudaMemcpyAsync(dst[q], src[q], bytes, cudaMemcpyDeviceToDevice, m->stream));
    return BH_OK;
}

// ------------------------------------------------------------- autotuner
//
// The launch configuration of the stepping kernels: G, the shots of one
// launch group (one launch, or one cooperative phase, covers the tiles of G
// shots; small groups keep a group's window state in L2, large ones give a
// launch more tiles to overlap), the launch form (2: cooperative when a
// group's tiles fit the co-resident blocks, else one launch per half-step;
// 0: always per half-step; 1: always cooperative), and the forward tile
// code variant.  bh_tune times the candidates on the model and keeps the
// fastest; a cache file maps a key (GPU name, nr, window pitch, shots) to
// the choice.

std::string tune_key(const char* gpu, int nr, int P, int nshots)
{
    std::string name(gpu);
    for (char& c : name)
        if (c == ' ' || c == '\t' || c == '|') c = '_';
    char buf[96];
    snprintf(buf, sizeof buf, "|nr%d|P%d|shots%d", nr, P, nshots);
    return name + buf;
}

// the last line of the cache with this key:
// "<key> <G> <form> <tile code> <split> <tile order> ..."
bool tune_lookup(const char* path, const std::string& key, int* G, int* form, int* code,
                 int* split, int* order)
{
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::istringstream is(line);
        std::string k;
        int g = 0, p = -1, v = -1, sp = -1, od = -1;
        std::string rest;
        if (!(is >> k >> g >> p >> v >> sp >> od >> rest)) continue;
        if (k != key || g < 1 || g > kGroup || p < 0 || p > 2 || v < 0 || v > 1 || sp < 0 ||
            sp > 4 || od < 0 || od > 1)
            continue;
        *G = g;
        *form = p;
        *code = v;
        *split = sp;
        *order = od;
        found = true;
    }
    return found;
}

bh_status set_group(bh_model* m, int G)
{
    if (G < 1 || G > std::min(kGroup, m->nshots))
        return fail(m, BH_ERR_INVALID_ARG, "group must be in [1, min(32, nshots)]");
    if (G == m->G) return BH_OK;
    m->G = G;
    m->have_forward = m->have_gradient = false;
    ++m->state_version;
    return build_tiles(m);
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
    if (g.snapshot_precision < 0 || g.snapshot_precision > 2)
        return fail(nullptr, BH_ERR_INVALID_ARG, "snapshot_precision must be 0, 1 or 2");
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
    m->G = std::min(nshots, kGroup);
    // a window's own loads reach 3 columns past its end, plus the copy shift
    m->Pw = (nz_global + 8 + 31) / 32 * 32;
    m->stream = (cudaStream_t)stream;
    m->snap_prec = g.snapshot_precision;
    const int nr = g.nr;
    const size_t ng = (size_t)nr * nz_global;
    const size_t pl = plane(m);

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
    // history window and checkpoints
    if (g.checkpoint_cap_bytes == 0) {
        m->L = g.nt;  // store every step
        m->nsnap = 0;
        m->tail = g.nt;
        m->n_tail0 = 0;
        m->hist_slots = g.nt + 1;
        m->recompute_steps = 0;
    } else {
        bh_status st = plan_checkpoints(m, g.checkpoint_cap_bytes);
        if (st != BH_OK) return bail(st);
    }
    CK(dalloc(&m->d_lam, ng));
    CK(dalloc(&m->d_mu, ng));
    CK(dalloc(&m->d_rho, ng));
    CK(dalloc(&m->d_vp, ng));
    CK(dalloc(&m->d_vs, ng));
    CK(dalloc(&m->d_bvr, ng));
    CK(dalloc(&m->d_bvz, ng));
    CK(dalloc(&m->d_muh, ng));
    CK(dalloc(&m->d_mask, ng));
    CK(dalloc(&m->d_colcov, (size_t)nz_global));
    CK(dalloc(&m->d_rprof, 6 * (size_t)nr));
    CK(dalloc(&m->d_fwd, (size_t)nshots * kFwdPlanes * pl));
    CK(dalloc(&m->d_fwd2, (size_t)nshots * kFields * pl));
    CK(dalloc(&m->d_adj, (size_t)nshots * kAdjPlanes * pl));
    CK(dalloc(&m->d_wcoef, (size_t)4 * 5 * nr * m->Pw));
    CK(dalloc(&m->d_hist, (size_t)nshots * m->hist_slots * 2 * pl));
    CK(dalloc((char**)&m->d_snap,
              (size_t)m->nsnap * nshots * kFwdPlanes * pl * (m->snap_prec ? 2 : 4)));
    CK(dalloc(&m->d_snap_max, (size_t)m->nsnap * nshots * kFwdPlanes));
    CK(dalloc(&m->d_Hg, 2 * ng));
    CK(dalloc(&m->d_scal, 16));
    CK(dalloc(&m->d_part, 8 * (size_t)kMaxParts));
    CK(dalloc(&m->d_bar, 4));
    m->tma_ok = encode_maps(m);
    {
        int dev = 0, sms = 0, coop = 0, nb = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        // the adjoint kernels want 5 blocks of ~42 KB shared memory per SM;
        // the forward kernels (14 KB per block) keep the default split, which
        // leaves L1 room for their read-only coefficient loads (the maximum
        // shared-memory carveout made them 9-23 % slower)
        const void* big_smem[] = {
            (const void*)k_adj_persist<1, true>,  (const void*)k_adj_persist<kGroup, true>,
            (const void*)k_adj_persist<1, false>, (const void*)k_adj_persist<kGroup, false>,
            (const void*)k_adj_stress<1, true>,   (const void*)k_adj_stress<kGroup, true>,
            (const void*)k_adj_stress<1, false>,  (const void*)k_adj_stress<kGroup, false>,
            (const void*)k_adj_vel<1, true>,      (const void*)k_adj_vel<kGroup, true>,
            (const void*)k_adj_vel<1, false>,     (const void*)k_adj_vel<kGroup, false>,
#define BH_CLASS_KERNELS(PM)                                                                    \
    (const void*)k_adj_stress_c<1, true, PM>, (const void*)k_adj_stress_c<kGroup, true, PM>,    \
        (const void*)k_adj_stress_c<1, false, PM>,                                              \
        (const void*)k_adj_stress_c<kGroup, false, PM>, (const void*)k_adj_vel_c<1, true, PM>,  \
        (const void*)k_adj_vel_c<kGroup, true, PM>, (const void*)k_adj_vel_c<1, false, PM>,     \
        (const void*)k_adj_vel_c<kGroup, false, PM>
            BH_CLASS_KERNELS(PM_INTERIOR), BH_CLASS_KERNELS(PM_PML)};
#undef BH_CLASS_KERNELS
        for (const void* f : big_smem)
            CK(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared));
        // the pipelined forward kernels hold two ~41 KB stages per block and
        // read nothing through L1 but the 1/r arrays
        const void* pipe[] = {(const void*)k_fwd_vel_pipe<1>, (const void*)k_fwd_vel_pipe<kGroup>,
                              (const void*)k_fwd_stress_pipe<1>,
                              (const void*)k_fwd_stress_pipe<kGroup>};
        m->pipe_blocks = 1 << 30;
        for (const void* f : pipe) {
            CK(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared));
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kThreads, 0));
            m->pipe_blocks = std::min(m->pipe_blocks, nb * sms);
        }
        // both forward variants are bounded to 5 blocks of 128 threads; the
        // smaller of their counts serves both
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fwd_persist<1, 0>, kThreads, 0));
        m->fwd_blocks = nb * sms;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fwd_persist<1, 1>, kThreads, 0));
        m->fwd_blocks = std::min(m->fwd_blocks, nb * sms);
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_persist<1, true>, kThreads, 0));
        m->adj_blocks = nb * sms;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_persist<1, false>, kThreads, 0));
        m->adj_blocks_nr = nb * sms;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_persist<kGroup, false>, kThreads,
                                                         0));
        m->adj_blocks_g_nr = nb * sms;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fwd_persist<kGroup, 0>, kThreads,
                                                         0));
        m->fwd_blocks_g = nb * sms;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fwd_persist<kGroup, 1>, kThreads,
                                                         0));
        m->fwd_blocks_g = std::min(m->fwd_blocks_g, nb * sms);
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_persist<kGroup, true>, kThreads,
                                                         0));
        m->adj_blocks_g = nb * sms;
        if (!coop || std::min(std::min(m->fwd_blocks, m->adj_blocks),
                              std::min(m->fwd_blocks_g, m->adj_blocks_g)) < 1 ||
            std::min(m->adj_blocks_nr, m->adj_blocks_g_nr) < 1)
            m->persistent = 0;
    }
    m->shots.resize(nshots);
    std::vector<uint8_t> colcov(nz_global, 0);
    for (int s = 0; s < nshots; ++s) {
        ShotHost& sd = m->shots[s];
        const bh_shot_desc& d = shots[s];
        sd.z0 = d.z_offset;
        sd.nz = d.nz;
        sd.src_ir = d.src_ir;
        sd.src_iz = d.src_iz;
        sd.nrec = d.nrec;
        sd.rec_iz.assign(d.rec_iz, d.rec_iz + d.nrec);
        for (int j = g.npml_z; j < d.nz - g.npml_z; ++j) colcov[d.z_offset + j] = 1;
    }
    CK(cudaMemcpyAsync(m->d_colcov, colcov.data(), nz_global, cudaMemcpyHostToDevice,
                       m->stream));
    CK(cudaStreamSynchronize(m->stream));
#undef CK
    bh_status st = load_model(m, vp, vs, rho, true);
    if (st != BH_OK) return bail(st);
    st = setup_profiles(m);
    if (st != BH_OK) return bail(st);
    st = setup_shots(m);
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
    const size_t pl = plane(m);
    const size_t seis_per_shot = (size_t)m->nrec_max * gd.nt;
    m->have_forward = m->have_gradient = false;
    ++m->state_version;
    m->runs_fwd = 0;
    for (int s = 0; s < m->nshots; ++s) {
        m->h_shots[s].q.wavelet = wavelet;
        m->h_shots[s].q.seis = seis + seis_per_shot * s;
    }
    BH_CUDA(m, cudaMemsetAsync(seis, 0, seis_per_shot * m->nshots * sizeof(float), m->stream));
    BH_CUDA(m, cudaMemsetAsync(m->d_fwd, 0, (size_t)m->nshots * kFwdPlanes * pl * sizeof(float),
                               m->stream));
    BH_CUDA(m, cudaMemsetAsync(m->d_fwd2, 0, (size_t)m->nshots * kFields * pl * sizeof(float),
                               m->stream));
    // sweep once, recording: take the schedule's first snapshots on the way
    // through the segments, then store the tail's history as it goes (all of
    // it when every step is stored)
    int n = 0;
    for (const auto& sp : m->spine) {
        const int n1 = std::min(m->n_tail0, sp.first * m->L);
        BH_TRY(run_forward(m, n, n1, -1, true, &m->runs_fwd));
        n = n1;
        BH_TRY(snapshot(m, sp.second, true));
    }
    BH_TRY(run_forward(m, n, m->n_tail0, -1, true, &m->runs_fwd));
    BH_TRY(run_forward(m, m->n_tail0, gd.nt, m->n_tail0, true, &m->runs_fwd));
    BH_LAUNCH(m);
    m->have_forward = true;
    return BH_OK;
}

bh_status bh_residual_misfit(bh_model* m, const float* seis_mod, const float* seis_obs,
                             float* resid, double* J)
{
    if (!m || !seis_mod || !seis_obs || !resid || !J)
        return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    const size_t n = (size_t)m->nshots * m->nrec_max * m->grid.nt;
    k_misfit<<<1, kRedThreads, 0, m->stream>>>(n, seis_mod, seis_obs, resid, m->d_scal);
    BH_KERNEL(m);
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
    const size_t pl = plane(m);
    const size_t ng = (size_t)gd.nr * m->nzg;
    const size_t seis_per_shot = (size_t)m->nrec_max * gd.nt;
    m->runs_adj = 0;
    m->adj_rho = g_rho != nullptr;
    for (int s = 0; s < m->nshots; ++s) m->h_shots[s].a.resid = resid + seis_per_shot * s;
    BH_CUDA(m, cudaMemsetAsync(g_lam, 0, ng * sizeof(double), m->stream));
    BH_CUDA(m, cudaMemsetAsync(g_mu, 0, ng * sizeof(double), m->stream));
    if (g_rho) BH_CUDA(m, cudaMemsetAsync(g_rho, 0, ng * sizeof(double), m->stream));
    BH_CUDA(m, cudaMemsetAsync(m->d_Hg, 0, 2 * ng * sizeof(double), m->stream));
    BH_CUDA(m, cudaMemsetAsync(m->d_adj, 0, (size_t)m->nshots * kAdjPlanes * pl * sizeof(float),
                               m->stream));
    for (int s = 0; s < m->nshots; ++s) {
        k_adj_inject<<<(m->shots[s].nz + 127) / 128, 128, 0, m->stream>>>(m->h_shots[s], gd.nt - 1);
        BH_KERNEL(m);
    }
    // the tail first: its history is the sweep's own
    BH_TRY(run_adjoint(m, m->n_tail0, gd.nt, m->n_tail0, &m->runs_adj));
    for (const Act& a : m->plan) {
        switch (a.kind) {
        case ACT_RESTORE: BH_TRY(snapshot(m, a.a, false)); break;
        case ACT_TAKE: BH_TRY(snapshot(m, a.a, true)); break;
        case ACT_ADVANCE:
            BH_TRY(run_forward(m, a.a * m->L, std::min(m->n_tail0, a.b * m->L), -1, false,
                               &m->runs_adj));
            break;
        case ACT_REVERSE: {
            // refill the window with the segment's history, then reverse it
            const int n0 = a.a * m->L, n1 = std::min(m->n_tail0, n0 + m->L);
            BH_TRY(run_forward(m, n0, n1, n0, false, &m->runs_adj));
            BH_TRY(run_adjoint(m, n0, n1, n0, &m->runs_adj));
            break;
        }
        }
    }
    FinK f;
    f.g_lam = g_lam;
    f.g_mu = g_mu;
    f.g_rho = g_rho;
    f.H_lam = m->d_Hg;
    f.H_mu = m->d_Hg + ng;
    const dim3 blk = block2d();
    for (int s = 0; s < m->nshots; ++s) {
        k_finalize<<<grid2d(gd.nr, m->shots[s].nz), blk, 0, m->stream>>>(m->h_shots[s], f);
        BH_KERNEL(m);
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
    const int np = parts_for(ng);
    k_masked_max2_part<<<np, kPartThreads, 0, m->stream>>>(ng, m->d_mask, m->d_Hg, m->d_Hg + ng,
                                                           m->d_part);
    BH_KERNEL(m);
    k_masked_max2_finish<<<1, kPartThreads, 0, m->stream>>>(m->d_part, np, m->d_scal + 2);
    BH_KERNEL(m);
    k_precondition<<<(unsigned)((ng + 255) / 256), 256, 0, m->stream>>>(
        ng, m->d_mask, m->d_Hg, m->d_Hg + ng, m->d_scal + 2, eps_rel, g_lam, g_mu);
    BH_KERNEL(m);
    return BH_OK;
}

bh_status bh_update(bh_model* m, const double* g_lam, const double* g_mu, double kappa,
                    double* alpha_out, float* vp_out, float* vs_out)
{
    if (!m || !g_lam || !g_mu) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    if (!(kappa >= 0.0)) return fail(m, BH_ERR_INVALID_ARG, "kappa must be >= 0");
    const size_t ng = (size_t)m->grid.nr * m->nzg;
    const int np = parts_for(ng);
    k_update_alpha_part<<<np, kPartThreads, 0, m->stream>>>(ng, m->d_mask, m->d_lam, m->d_mu,
                                                            g_lam, g_mu, m->d_part);
    BH_KERNEL(m);
    k_update_alpha_finish<<<1, kPartThreads, 0, m->stream>>>(m->d_part, np, kappa,
                                                             m->d_scal + 4);
    BH_KERNEL(m);
    const unsigned nb = (unsigned)((ng + 255) / 256);
    k_update_apply<<<nb, 256, 0, m->stream>>>(ng, m->d_mask, g_lam, g_mu, m->d_scal + 4,
                                             m->d_rho, m->d_lam, m->d_mu, m->d_vp, m->d_vs);
    BH_KERNEL(m);
    BH_TRY(rebuild_coefficients(m));
    BH_TRY(copy_model_out(m, vp_out, vs_out, nullptr));
    if (alpha_out) {
        BH_CUDA(m, cudaMemcpyAsync(alpha_out, m->d_scal + 4, 2 * sizeof(double),
                                   cudaMemcpyDeviceToHost, m->stream));
        BH_CUDA(m, cudaStreamSynchronize(m->stream));
    }
    m->have_forward = m->have_gradient = false;
    ++m->state_version;
    return BH_OK;
}

bh_status bh_update_velocity(bh_model* m, const double* g_lam, const double* g_mu,
                             const double* g_rho, int update_rho, double kappa, double* alpha_out,
                             float* vp_out, float* vs_out, float* rho_out)
{
    if (!m || !g_lam || !g_mu) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    if (!(kappa >= 0.0)) return fail(m, BH_ERR_INVALID_ARG, "kappa must be >= 0");
    if (update_rho != 0 && update_rho != 1)
        return fail(m, BH_ERR_INVALID_ARG, "update_rho must be 0 or 1");
    const size_t ng = (size_t)m->grid.nr * m->nzg;
    const int np = parts_for(ng);
    k_vupdate_part<<<np, kPartThreads, 0, m->stream>>>(ng, m->d_mask, m->d_vp, m->d_vs, m->d_rho,
                                                       g_lam, g_mu, g_rho, m->d_part);
    BH_KERNEL(m);
    k_vupdate_finish<<<1, kPartThreads, 0, m->stream>>>(m->d_part, np, kappa, update_rho,
                                                        m->d_scal + 8);
    BH_KERNEL(m);
    k_vupdate_apply<<<(unsigned)((ng + 255) / 256), 256, 0, m->stream>>>(
        ng, m->d_mask, g_lam, g_mu, g_rho, m->d_scal + 8, update_rho, m->d_vp, m->d_vs, m->d_rho,
        m->d_lam, m->d_mu);
    BH_KERNEL(m);
    BH_TRY(rebuild_coefficients(m));
    BH_TRY(copy_model_out(m, vp_out, vs_out, rho_out));
    if (alpha_out) {
        BH_CUDA(m, cudaMemcpyAsync(alpha_out, m->d_scal + 8, 3 * sizeof(double),
                                   cudaMemcpyDeviceToHost, m->stream));
        BH_CUDA(m, cudaStreamSynchronize(m->stream));
    }
    m->have_forward = m->have_gradient = false;
    ++m->state_version;
    return BH_OK;
}

bh_status bh_velocity_gradient(bh_model* m, const double* g_lam, const double* g_mu,
                               const double* g_rho, float* g_vp, float* g_vs, float* g_rho_v)
{
    if (!m || !g_lam || !g_mu) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    const size_t ng = (size_t)m->grid.nr * m->nzg;
    k_velocity_gradient<<<(unsigned)((ng + 255) / 256), 256, 0, m->stream>>>(
        ng, m->d_vp, m->d_vs, m->d_rho, g_lam, g_mu, g_rho, g_vp, g_vs, g_rho_v);
    BH_KERNEL(m);
    return BH_OK;
}

bh_status bh_get_model(bh_model* m, float* vp, float* vs)
{
    if (!m || !vp || !vs) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    return copy_model_out(m, vp, vs, nullptr);
}

bh_status bh_get_density(bh_model* m, float* rho)
{
    if (!m || !rho) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    return copy_model_out(m, nullptr, nullptr, rho);
}

bh_status bh_set_option(bh_model* m, const char* key, double value)
{
    if (!m || !key) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    const std::string k(key);
    if (k == "persistent") {
        if (value != 0.0 && value != 1.0 && value != 2.0)
            return fail(m, BH_ERR_INVALID_ARG, "persistent must be 0, 1 or 2");
        if (value != 0.0 && std::min(std::min(m->fwd_blocks, m->adj_blocks),
                                     std::min(m->fwd_blocks_g, m->adj_blocks_g)) < 1)
            return fail(m, BH_ERR_UNSUPPORTED, "cooperative launch not available");
        m->persistent = (int)value;
    } else if (k == "split") {
        if (value != 0.0 && value != 1.0 && value != 2.0 && value != 3.0 && value != 4.0)
            return fail(m, BH_ERR_INVALID_ARG, "split must be 0 .. 4");
        if (value == 4.0 && !m->tma_ok)
            return fail(m, BH_ERR_UNSUPPORTED, "tensor maps could not be encoded");
        if (value == 2.0 && m->pipe_blocks < 1)
            return fail(m, BH_ERR_UNSUPPORTED, "the pipelined kernels do not fit an SM");
        m->split = (int)value;
    } else if (k == "tile_order") {
        if (value != 0.0 && value != 1.0)
            return fail(m, BH_ERR_INVALID_ARG, "tile_order must be 0 or 1");
        if ((int)value == m->tile_order) return BH_OK;
        m->tile_order = (int)value;
        return build_tiles(m);
    } else if (k == "pipe_grid") {
        if (value < 0.0 || value > 1e6 || value != std::floor(value))
            return fail(m, BH_ERR_INVALID_ARG, "pipe_grid must be an integer in [0, 1e6]");
        m->pipe_grid = (int)value;
    } else if (k == "tile_code") {
        if (value != 0.0 && value != 1.0)
            return fail(m, BH_ERR_INVALID_ARG, "tile_code must be 0 or 1");
        m->tile_code = (int)value;
    } else if (k == "group") {
        if (value != std::floor(value)) return fail(m, BH_ERR_INVALID_ARG, "group must be an integer");
        return set_group(m, (int)value);
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

bh_status bh_get_info(bh_model* m, const char* key, double* value)
{
    if (!m || !key || !value) return fail(m, BH_ERR_INVALID_ARG, "NULL argument");
    const std::string k(key);
    const size_t pl = plane(m), ng = (size_t)m->grid.nr * m->nzg;
    if (k == "history_steps") *value = m->L;
    else if (k == "tail_steps") *value = m->tail;
    else if (k == "snapshots") *value = m->nsnap;
    else if (k == "recompute_steps") *value = (double)m->recompute_steps;
    else if (k == "tiles") *value = m->ntiles;
    else if (k == "persistent_runs_per_step") *value = (double)(m->runs_fwd + m->runs_adj);
    else if (k == "persistent_blocks_fwd") *value = m->fwd_blocks;
    else if (k == "persistent_blocks_adj") *value = m->adj_blocks;
    else if (k == "persistent") *value = m->persistent;
    else if (k == "history_snapshot_bytes")
        *value = (double)pl * sizeof(float) * m->nshots *
                 (2.0 * m->hist_slots + (double)m->nsnap * kFwdPlanes * (m->snap_prec ? 0.5 : 1.0));
    else if (k == "snapshot_precision") *value = m->snap_prec;
    else if (k == "kernel_launches") *value = (double)m->launches;
    else if (k == "state_version") *value = (double)m->state_version;
    else if (k == "group") *value = m->G;
    else if (k == "tile_code") *value = m->tile_code;
    else if (k == "split") *value = m->split;
    else if (k == "pipe_grid") *value = m->pipe_grid;
    else if (k == "tile_order") *value = m->tile_order;
    else if (k == "tma") *value = m->tma_ok ? 1.0 : 0.0;
    else if (k == "pipe_blocks") *value = m->pipe_blocks;
    else if (k == "device_bytes")
        *value = (double)pl * sizeof(float) * m->nshots *
                     (kFwdPlanes + kFields + kAdjPlanes + 2.0 * m->hist_slots) +
                 20.0 * m->grid.nr * m->Pw * sizeof(float) +
                 (double)pl * (m->snap_prec ? 2 : 4) * m->nshots * m->nsnap * kFwdPlanes +
                 (double)ng * (6 * sizeof(float) + 1 + 2 * sizeof(double));
    else return fail(m, BH_ERR_INVALID_ARG, "unknown key " + k);
    return BH_OK;
}

bh_status bh_checkpoint_plan(int nseg, int nsnap, int* actions, int max_actions,
                             int* n_actions, int* spine, int max_spine, int* n_spine)
{
    if (nseg < 1 || nsnap < 0 || !actions || !n_actions || !spine || !n_spine)
        return fail(nullptr, BH_ERR_INVALID_ARG, "bad argument");
    std::vector<Act> plan;
    std::vector<std::pair<int, int>> sp;
    long long adv = 0;
    build_plan(nseg, nsnap, &plan, &sp, &adv);
    *n_actions = (int)plan.size();
    *n_spine = (int)sp.size();
    if ((int)plan.size() > max_actions || (int)sp.size() > max_spine)
        return fail(nullptr, BH_ERR_INVALID_ARG, "output arrays too small");
    for (size_t k = 0; k < plan.size(); ++k) {
        actions[3 * k] = plan[k].kind;
        actions[3 * k + 1] = plan[k].a;
        actions[3 * k + 2] = plan[k].b;
    }
    for (size_t k = 0; k < sp.size(); ++k) {
        spine[2 * k] = sp[k].first;
        spine[2 * k + 1] = sp[k].second;
    }
    return BH_OK;
}

bh_status bh_tune_lookup(const char* cache_path, const char* gpu_name, int nr, int window_pitch,
                         int nshots, int* group, int* form, int* tile_code, int* split,
                         int* tile_order)
{
    if (!cache_path || !gpu_name || !group || !form || !tile_code || !split || !tile_order)
        return fail(nullptr, BH_ERR_INVALID_ARG, "bh_tune_lookup: NULL argument");
    if (!tune_lookup(cache_path, tune_key(gpu_name, nr, window_pitch, nshots), group, form,
                     tile_code, split, tile_order))
        return fail(nullptr, BH_ERR_STATE, "bh_tune_lookup: no entry for this key");
    return BH_OK;
}

bh_status bh_tune(bh_model* m, int steps, const char* cache_path, char* choice, int choice_len)
{
    if (!m || steps < 1) return fail(m, BH_ERR_INVALID_ARG, "bad argument");
    int dev = 0;
    BH_CUDA(m, cudaGetDevice(&dev));
    cudaDeviceProp prop;
    BH_CUDA(m, cudaGetDeviceProperties(&prop, dev));
    const std::string key = tune_key(prop.name, m->grid.nr, m->P, m->nshots);
    const bool coop = std::min(std::min(m->fwd_blocks, m->adj_blocks),
                               std::min(m->fwd_blocks_g, m->adj_blocks_g)) >= 1;
    int bestG = m->G, bestForm = m->persistent, bestCode = m->tile_code, bestSplit = m->split;
    int bestOrder = m->tile_order;
    double best_ms = -1.0;
    std::string how = "cached";
    if (!(cache_path &&
          tune_lookup(cache_path, key, &bestG, &bestForm, &bestCode, &bestSplit, &bestOrder))) {
        const int S = std::min(std::min(steps, m->grid.nt), m->hist_slots - 1);
        if (S < 1) return fail(m, BH_ERR_STATE, "history window too short to time a step");
        // inputs the timed runs read: a zero wavelet and residual
        const size_t nbuf = std::max((size_t)m->nshots * m->nrec_max * m->grid.nt,
                                     (size_t)m->grid.nt);
        float* zero = nullptr;
        BH_CUDA(m, dalloc(&zero, nbuf));
        BH_CUDA(m, cudaMemsetAsync(zero, 0, nbuf * sizeof(float), m->stream));
        for (int sh = 0; sh < m->nshots; ++sh) {
            m->h_shots[sh].q.wavelet = zero;
            m->h_shots[sh].q.seis = zero;
            m->h_shots[sh].a.resid = zero;
        }
        const bool rho_saved = m->adj_rho;
        m->adj_rho = false;
        cudaEvent_t e0, e1;
        BH_CUDA(m, cudaEventCreate(&e0));
        BH_CUDA(m, cudaEventCreate(&e1));
        std::vector<int> Gs;
        for (int g = 1; g <= std::min(kGroup, m->nshots); g *= 2) Gs.push_back(g);
        if (m->nshots <= kGroup && Gs.back() != m->nshots) Gs.push_back(m->nshots);
        char line[160];
        std::string log;
        bh_status st = BH_OK;
        for (int code = 0; code <= 1 && st == BH_OK; ++code)
        for (int g : Gs) {
            m->tile_code = code;
            if ((st = set_group(m, g)) != BH_OK) break;
            // the launch forms that differ for this grouping
            int fit = 0;
            const int ng = (int)m->group_ntiles.size();
            for (int grp = 0; grp < ng; ++grp) {
                m->persistent = 2;
                fit += persistent_for(m, grp, false) && persistent_for(m, grp, true);
            }
            std::vector<int> forms = {0};
            if (coop) {
                forms.push_back(1);
                if (fit > 0 && fit < ng) forms.push_back(2);
            }
            for (int f : forms)
            for (int sp = 0; sp <= (f != 0 ? 0 : code == 1 ? 4 : 1); ++sp)
            for (int od = 0; od <= (f != 0 ? 0 : 1) && st == BH_OK; ++od) {
                if ((sp == 2 && m->pipe_blocks < 1) || (sp == 4 && !m->tma_ok)) continue;
                m->persistent = f;
                m->split = sp;
                if (od != m->tile_order) {
                    m->tile_order = od;
                    if ((st = build_tiles(m)) != BH_OK) break;
                }
                float ms = 0.f;
                long long runs = 0;
                // the best of three runs after a warm-up
                float best_rep = -1.f;
                for (int rep = 0; rep < 4 && st == BH_OK; ++rep) {
                    cudaEventRecord(e0, m->stream);
                    if ((st = run_forward(m, 0, S, 0, false, &runs)) != BH_OK) break;
                    if ((st = run_adjoint(m, 0, S, 0, &runs)) != BH_OK) break;
                    cudaEventRecord(e1, m->stream);
                    if (cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                        st = fail(m, BH_ERR_CUDA, "bh_tune: event timing failed");
                    if (rep > 0 && (best_rep < 0.f || ms < best_rep)) best_rep = ms;
                }
                ms = best_rep;
                if (st != BH_OK) break;
                snprintf(line, sizeof line, "%scode=%d G=%d form=%d split=%d order=%d %.3f ms",
                         log.empty() ? "" : "; ", code, g, f, sp, od, ms);
                log += line;
                if (best_ms < 0 || ms < best_ms) {
                    best_ms = ms;
                    bestG = g;
                    bestForm = f;
                    bestCode = code;
                    bestSplit = sp;
                    bestOrder = od;
                }
            }
            if (st != BH_OK) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        m->adj_rho = rho_saved;
        cudaStreamSynchronize(m->stream);
        cudaFree(zero);
        if (st != BH_OK) return st;
        snprintf(line, sizeof line, "timed %d forward + %d adjoint steps per candidate: ", S, S);
        how = line + log;
        if (cache_path) {
            std::ofstream f(cache_path, std::ios::app);
            if (f) f << key << " " << bestG << " " << bestForm << " " << bestCode << " "
                     << bestSplit << " " << bestOrder << " " << best_ms << " ms/" << S
                     << "-step-pair\n";
        }
    }
    BH_TRY(set_group(m, bestG));
    if (bestForm != 0 && !coop) bestForm = 0;
    m->persistent = bestForm;
    m->tile_code = bestCode;
    m->split = (bestSplit == 2 && m->pipe_blocks < 1) || (bestSplit == 4 && !m->tma_ok) ? 1
                                                                                    : bestSplit;
    if (bestOrder != m->tile_order) {
        m->tile_order = bestOrder;
        BH_TRY(build_tiles(m));
    }
    m->have_forward = m->have_gradient = false;
    ++m->state_version;
    if (choice && choice_len > 0) {
        std::string txt = "group " + std::to_string(bestG) + ", form " +
                          std::to_string(bestForm) + ", tile code " + std::to_string(bestCode) +
                          ", split " + std::to_string(bestSplit) + ", tile order " +
                          std::to_string(bestOrder) + " (" + how + ")";
        snprintf(choice, (size_t)choice_len, "%s", txt.c_str());
    }
    return BH_OK;
}

bh_status bh_starting_model(int nr, int nz, double dr, double r_wall, double r_far,
                            const float* vp_wall, const float* vs_wall, const float* vp_far,
                            const float* vs_far, float vp_fluid, float* vp, float* vs,
                            void* stream)
{
    if (nr < 1 || nz < 1 || !(dr > 0) || !(r_wall >= 0) || !(r_far > r_wall) || !vp_wall ||
        !vs_wall || !vp_far || !vs_far || !vp || !vs)
        return fail(nullptr, BH_ERR_INVALID_ARG, "bh_starting_model: bad argument");
    const cudaStream_t st = (cudaStream_t)stream;
    k_starting_model<<<grid2d(nr, nz), block2d(), 0, st>>>(nr, nz, dr, r_wall, r_far, vp_wall,
                                                           vs_wall, vp_far, vs_far, vp_fluid,
                                                           vp, vs);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(nullptr, BH_ERR_CUDA, std::string("bh_starting_model: ") + cudaGetErrorString(e));
    return BH_OK;
}

bh_status bh_plan_history(int nt, double hist_step_bytes, double snapshot_bytes,
                          size_t cap_bytes, int* L, int* nsnap, int* tail, long long* recompute)
{
    if (nt < 1 || !(hist_step_bytes > 0) || !(snapshot_bytes > 0) || !L || !nsnap || !tail ||
        !recompute)
        return fail(nullptr, BH_ERR_INVALID_ARG, "bad argument");
    const HistPlan hp = choose_history_plan(nt, hist_step_bytes, snapshot_bytes, (double)cap_bytes);
    if (hp.recompute < 0)
        return fail(nullptr, BH_ERR_OOM, "cap too small for one history window");
    *L = hp.L;
    *nsnap = hp.nsnap;
    *tail = hp.tail;
    *recompute = hp.recompute;
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
    BH_TRY(bh_profile_read(m, 0, &t, &n));
    for (int k = 0; k < BH_KERNEL_COUNT; ++k) {
        m->prof_ms[k] = 0.0;
        m->prof_n[k] = 0;
    }
    return BH_OK;
}

}  // extern "C"
