// Device kernels of libbh: forward steps of Eq. 2, their exact transposes
// (the discrete adjoint of Eq. 6) with the correlations of Eq. 7 / Eq. 8
// fused in, and the per-shot finalisation.  FP32 stepping, Kahan-compensated
// FP32 gradient accumulation, FP64 per-cell results.
//
// Index conventions (window coordinates, z contiguous, row pitch P):
//   cell  (i,j): r=(i+1/2)dr, z=j dz        trr, ttt, tzz
//   v_r   (i,j): r=i dr,      z=j dz        v_r(0,.) = 0
//   v_z   (i,j): r=(i+1/2)dr, z=(j+1/2)dz
//   trz   (i,j): r=i dr,      z=(j+1/2)dz   trz(0,.) = 0
// Ghost values: half-r fields mirror evenly about the axis, integer-r fields
// oddly; everything beyond r >= nr or outside 0 <= z < nz is zero.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace bh {

constexpr float kC1 = 1.125f;              // 9/8
constexpr float kC2 = -0.041666666666666664f; // -1/24

struct WinK {
    int nr, nz, P;      // window rows, columns, row pitch of the state arrays
    int Pw;             // row pitch of the shared coefficient copies (CoefK w_*)
    int nzg, z0;        // global model pitch and the window's first global row
    int npml_r, npml_z;
    float dt, inv_dr, inv_dz;
};

struct CoefK {
    const float *lam, *mu, *rho;      // cells, global [nr][nzg]
    const float *bvr, *bvz, *muh;     // nodes, global [nr][nzg]
    const float *inv_r_int, *inv_r_half;          // [nr]
    const float *ar_int, *br_int, *ar_half, *br_half;  // radial C-PML [nr]
    const float *az_int, *bz_int, *az_half, *bz_half;  // axial C-PML of the window [nz]
    // lambda, mu (cells), harmonic mu (trz nodes), buoyancy at v_r and v_z
    // nodes of the global model, read through a copy shifted so that the
    // window's column 0 is 16-byte aligned: window node (i, j) is
    // w_*[i * Pw + j].  Several shots share one copy (one per z0 mod 4).
    // Beyond the window they hold the global model's neighbours, so staging
    // zero-fills outside 0 <= j < nz; at the window's last row the v_z
    // buoyancy and the trz harmonic mu follow the window's own rule instead
    // (bvz_at, muh_at), which the tiles with TILE_LAST patch in.
    const float *w_lam, *w_mu, *w_muh, *w_bvr, *w_bvz;
};

struct StateK {
    float *vr, *vz, *trr, *ttt, *tzz, *trz;
    float *psi[8];   // C-PML memories (forward) or adjoint memories, read side
    float *psi_w[8]; // write side (== psi in the forward; ping-pong in the adjoint)
};

// ---------------------------------------------------------------- loads

// field at half-r positions (cells, v_z): even mirror, zero outside
__device__ __forceinline__ float ld_h(const float* __restrict__ f, int i, int j, const WinK& g)
{
    if (j < 0 || j >= g.nz) return 0.f;
    if (i < 0) i = -1 - i;
    if (i >= g.nr) return 0.f;
    return f[(size_t)i * g.P + j];
}

// field at integer-r positions (v_r, trz): odd mirror, zero on the axis and outside
__device__ __forceinline__ float ld_i(const float* __restrict__ f, int i, int j, const WinK& g)
{
    if (j < 0 || j >= g.nz) return 0.f;
    float s = 1.f;
    if (i < 0) { i = -i; s = -1.f; }
    if (i == 0 || i >= g.nr) return 0.f;
    return s * f[(size_t)i * g.P + j];
}

__device__ __forceinline__ float d4(float p1, float m1, float p3, float m3)
{
    // c1 (f(+1/2) - f(-1/2)) + c2 (f(+3/2) - f(-3/2))
    return kC1 * (p1 - m1) + kC2 * (p3 - m3);
}

// buoyancy at v_z (i,j) and harmonic mu at trz (i,j) with the window's own
// axial edge: the last row sees only its own cells.
__device__ __forceinline__ float bvz_at(const CoefK& C, const WinK& g, int i, int j)
{
    size_t cg = (size_t)i * g.nzg + g.z0 + j;
    if (j == g.nz - 1) return 1.f / C.rho[cg];
    return C.bvz[cg];
}

__device__ __forceinline__ float muh_at(const CoefK& C, const WinK& g, int i, int j)
{
    size_t cg = (size_t)i * g.nzg + g.z0 + j;
    if (j == g.nz - 1) {
        float a = C.mu[cg - g.nzg], b = C.mu[cg];
        if (a <= 0.f || b <= 0.f) return 0.f;
        return 2.f / (1.f / a + 1.f / b);
    }
    return C.muh[cg];
}

// ------------------------------------------------------------- tiling
//
// Every stepping kernel works on tiles of kTR x kTZ nodes (16 rows of r by
// 32 columns of z).  A block has 128 threads, 8 column groups x 16 rows:
// each thread computes 4 consecutive z nodes of one row, with float4 loads
// and stores.  The block first stages what the tile's stencils read, rows
// i0-2 .. i0+17 and columns j0-4 .. j0+35 (16-byte aligned), into shared
// memory with the axis mirror and the zero edges applied; the stencils then
// read float4 rows of the staged tiles.  The adjoint tiles also build the
// transposed-stencil coefficients once per staged node.  Tiles that touch no
// C-PML layer (flag in the tile table) skip every layer branch.
//
// The same tile functions serve two launch forms: one kernel per half-step
// (one tile per block), and one persistent cooperative kernel per run, with a
// bounded grid barrier between half-steps.  State written inside a launch is
// read with ld.global.cg (L2, not the SM-private L1, which other SMs' writes
// do not update).
constexpr int kTZ = 32, kTR = 16, kH = 2;
constexpr int kSR = kTR + 2 * kH;  // staged rows
constexpr int kSZ = kTZ + 8;       // staged columns j0-4 .. j0+35
constexpr int kQ = kSZ / 4;        // float4 per staged row
constexpr int kThreads = 128;
typedef float Tile[kSR][kSZ];

enum {
    TILE_PML = 1,   // tile or halo touches a C-PML layer
    TILE_LAST = 2   // the staged columns hold the window's last node row
};

// Tile class: interior tiles or C-PML tiles.  A tile function compiled per
// class runs interior tiles without any layer state (fewer live registers,
// no layer branches); PM_ANY compiles one code path that reads the tile's
// flag.  The adjoint kernels always branch on the flag to the per-class
// instantiations; the forward kernels come in both variants (tile code 0:
// one path, 1: per class), chosen per model (option "tile_code", the
// autotuner): the per-class code is faster where the state stays in L2,
// the single path where it streams from HBM.  Every launch form of one
// variant runs the same arithmetic on every tile and agrees bit for bit;
// the two variants differ in the compiler's contraction of multiply-adds
// (rounding level).
enum { PM_INTERIOR = 0, PM_PML = 1, PM_ANY = 2 };

template <int PM>
__device__ __forceinline__ bool tile_pml(int flags)
{
    return PM == PM_ANY ? (flags & TILE_PML) != 0 : PM == PM_PML;
}

// Programmatic dependent launch: a kernel may be scheduled while its
// predecessor drains; it must wait here before touching the predecessor's
// outputs.  No-op when launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

// 4 consecutive floats (16-byte aligned) of a row
struct V4 {
    float v[4];
};

__device__ __forceinline__ V4 ld4cg(const float* p)
{
    const float4 t = __ldcg(reinterpret_cast<const float4*>(p));
    return V4{{t.x, t.y, t.z, t.w}};
}

// read-only data (model planes): non-coherent path
__device__ __forceinline__ V4 ld4g(const float* p)
{
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    return V4{{t.x, t.y, t.z, t.w}};
}

__device__ __forceinline__ V4 lds4(const Tile& s, int rr, int cc)
{
    const float4 t = *reinterpret_cast<const float4*>(&s[rr][cc]);
    return V4{{t.x, t.y, t.z, t.w}};
}

// 12 consecutive staged values of row rr from column cc (z neighbours)
struct V12 {
    float v[12];
};

__device__ __forceinline__ V12 lds12(const Tile& s, int rr, int cc)
{
    V12 r;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 t = *reinterpret_cast<const float4*>(&s[rr][cc + 4 * k]);
        r.v[4 * k] = t.x;
        r.v[4 * k + 1] = t.y;
        r.v[4 * k + 2] = t.z;
        r.v[4 * k + 3] = t.w;
    }
    return r;
}

// store 4 nodes of a row, columns j .. j+3, only those below nz
__device__ __forceinline__ void st4(float* p, int j, int nz, const float (&x)[4])
{
    if (j + 3 < nz) {
        *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (j + e < nz) p[e] = x[e];
    }
}

__device__ __forceinline__ void st4f2(float2* p, int j, int nz, const float2 (&x)[4])
{
    if (j + 3 < nz) {
        reinterpret_cast<float4*>(p)[0] = make_float4(x[0].x, x[0].y, x[1].x, x[1].y);
        reinterpret_cast<float4*>(p)[1] = make_float4(x[2].x, x[2].y, x[3].x, x[3].y);
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (j + e < nz) p[e] = x[e];
    }
}

__device__ __forceinline__ void ld4f2(const float2* p, float2 (&x)[4])
{
    const float4 a = __ldcg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldcg(reinterpret_cast<const float4*>(p) + 1);
    x[0] = make_float2(a.x, a.y);
    x[1] = make_float2(a.z, a.w);
    x[2] = make_float2(b.x, b.y);
    x[3] = make_float2(b.z, b.w);
}

// Staging: rows i0-2 .. i0+17, columns j0-4 .. j0+35 of a window field go
// into a Tile.  EVEN: half-r field (cells, v_z), mirror f[-1-k] = f[k].
// ODD: integer-r field (v_r, trz), f[-k] = -f[k], f[0] = 0.  ABS: integer-r
// coefficient (harmonic mu), f[-k] = f[k], zero on the axis.  Zero beyond nr
// and outside 0 <= z < nz.  The geometry of a staged float4 (a Slot) is the
// same for every field of a tile, so it is computed once and every field's
// load goes through it.
enum { EVEN = 0, ODD = 1, ABS = 2 };

struct Slot {
    int rr, cq;  // staged row, first staged column
    int off_e;   // plane offset of the even-mirrored source row, -1: zero
    int off_o;   // plane offset of the odd/abs-mirrored source row, -1: zero
    int offw_e, offw_o;  // the same in the coefficient copies (pitch Pw)
    int zlim;    // source floats inside 0 <= z < nz (4: all of them)
    bool neg;    // the row is a mirror image (odd fields change sign)
};

__device__ __forceinline__ int tid_of() { return threadIdx.y * 8 + threadIdx.x; }

__device__ __forceinline__ Slot slot_of(int it, int i0, int j0, const WinK& g)
{
    Slot s;
    s.rr = it / kQ;
    s.cq = 4 * (it - s.rr * kQ);
    const int i = i0 - kH + s.rr, j = j0 - 4 + s.cq;
    const bool zin = j >= 0 && j < g.nz;
    s.zlim = zin ? min(4, g.nz - j) : 0;
    const int ie = i < 0 ? -1 - i : i;
    const int io = i < 0 ? -i : i;
    s.neg = i < 0;
    s.off_e = (zin && ie < g.nr) ? ie * g.P + j : -1;
    s.off_o = (zin && io >= 1 && io < g.nr) ? io * g.P + j : -1;
    s.offw_e = (zin && ie < g.nr) ? ie * g.Pw + j : -1;
    s.offw_o = (zin && io >= 1 && io < g.nr) ? io * g.Pw + j : -1;
    return s;
}

// Asynchronous staging (cp.async, 16 bytes per slot, through L2 only): the
// copy lands in the tile without passing through registers and zero-fills
// whatever lies outside the source (src-size below 16).  Odd fields then
// need their mirrored rows negated (negate_slot) after the wait.  POS: an
// integer-r field read only at rows i >= 1, not mirrored (zero elsewhere).
enum { POS = 3 };

__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// W: f is a shared coefficient copy (pitch Pw) rather than a window plane
template <int KIND, bool W = false>
__device__ __forceinline__ void stage_async(Tile& t, const float* __restrict__ f, const Slot& s)
{
    int off = W ? (KIND == EVEN ? s.offw_e : s.offw_o) : (KIND == EVEN ? s.off_e : s.off_o);
    if (KIND == POS && s.neg) off = -1;
    const float* src = f + (off >= 0 ? off : 0);
    const unsigned bytes = off >= 0 ? 4u * (unsigned)s.zlim : 0u;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(&t[s.rr][s.cq])),
                 "l"(src), "r"(bytes)
                 : "memory");
}

// this thread's copies have landed (other threads' need a __syncthreads)
__device__ __forceinline__ void async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void negate_slot(Tile& t, const Slot& s)
{
    float4* p = reinterpret_cast<float4*>(&t[s.rr][s.cq]);
    float4 v = *p;
    v.x = -v.x;
    v.y = -v.y;
    v.z = -v.z;
    v.w = -v.w;
    *p = v;
}

// slot of the staged region that is one of the tile's own float4 groups
__device__ __forceinline__ bool own_slot(const Slot& s)
{
    return s.rr >= kH && s.rr < kH + kTR && s.cq >= 4 && s.cq < 4 + kTZ;
}

// C-PML profiles of a tile's staged region, read from shared memory by the
// layer branches (the profile arrays would otherwise come from L2 on every
// slot: L1 is small next to the staged tiles).  r: per staged row, a and b
// of the half-r profile at the even-mirrored row and of the integer-r
// profile at row |i|; z: per staged column, the axial a and b at integer
// and half positions (zero outside 0 <= z < nz).
struct __align__(16) Prof {
    float r[4][kSR];  // ar_half, br_half (even row), ar_int, br_int (|i|)
    float z[4][kSZ];  // az_int, bz_int, az_half, bz_half
};

__device__ __forceinline__ void stage_prof(Prof& p, const CoefK& C, const WinK& g, int i0, int j0)
{
    const int tid = tid_of();
    if (tid < kSR) {
        const int i = i0 - kH + tid;
        const int ie = i < 0 ? -1 - i : i, io = i < 0 ? -i : i;
        p.r[0][tid] = ie < g.nr ? __ldg(C.ar_half + ie) : 0.f;
        p.r[1][tid] = ie < g.nr ? __ldg(C.br_half + ie) : 0.f;
        p.r[2][tid] = io < g.nr ? __ldg(C.ar_int + io) : 0.f;
        p.r[3][tid] = io < g.nr ? __ldg(C.br_int + io) : 0.f;
    } else if (tid >= 32 && tid < 32 + kSZ) {
        const int cz = tid - 32, j = j0 - 4 + cz;
        const bool in = j >= 0 && j < g.nz;
        p.z[0][cz] = in ? __ldg(C.az_int + j) : 0.f;
        p.z[1][cz] = in ? __ldg(C.bz_int + j) : 0.f;
        p.z[2][cz] = in ? __ldg(C.az_half + j) : 0.f;
        p.z[3][cz] = in ? __ldg(C.bz_half + j) : 0.f;
    }
}

__device__ __forceinline__ V4 prof4(const float* row, int cz)
{
    const float4 t = *reinterpret_cast<const float4*>(row + cz);
    return V4{{t.x, t.y, t.z, t.w}};
}

// own-node index helpers: thread (x = column group, y = row)
struct Own {
    int i, rr, j, cc, c;  // window row, staged row, first column, staged column, plane index
    int cw;               // index in the coefficient copies
    bool live;
};

__device__ __forceinline__ Own own_of(const WinK& g, int i0, int j0)
{
    Own o;
    o.i = i0 + threadIdx.y;
    o.rr = threadIdx.y + kH;
    o.j = j0 + 4 * threadIdx.x;
    o.cc = 4 * threadIdx.x + 4;
    o.live = o.i < g.nr && o.j < g.nz;
    o.c = o.i * g.P + o.j;
    o.cw = o.i * g.Pw + o.j;
    return o;
}

// Replace element j_last - j of a 4-node group starting at column j (if it
// lies there) by val: the window's last-row coefficients.
__device__ __forceinline__ void patch4(V4& x, int j, int j_last, float val)
{
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (j + e == j_last) x.v[e] = val;
}

// ------------------------------------------------- bounded grid barrier

struct BarK {
    unsigned* count;               // arrivals since the launch began (monotonic)
    int* err;                      // 1 once any wait gave up
    unsigned expected;             // arrivals that complete one barrier
    unsigned long long timeout_ns; // give up after this long
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// All blocks of a cooperative launch meet at every barrier; `epoch` counts
// the block's barriers (the same sequence in every block).  The barrier is
// split in two: grid_arrive publishes the block's writes with one
// release-acquire increment of a monotonic counter; grid_wait polls it with acquire loads
// until it reaches epoch * expected.  Between the two a block may do work
// that no other block reads in the next phase (its own accumulators), which
// then overlaps the barrier latency.  The wait is bounded twice, by the wall
// clock and by a poll count; when it runs out, or another block reports that
// it did, grid_wait returns false in every thread of the block, the caller
// returns from the kernel, and the host reads the error flag.  Writes before
// the arrival are visible to ld.global.cg loads and cp.async.cg copies after
// the wait.  Both halves are called by every thread of the block.
__device__ __forceinline__ void grid_arrive(const BarK& b, unsigned& epoch)
{
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        // an acq_rel atomic measured ~1 us faster per barrier than a
        // release reduction or a fence + relaxed atomic on GB300
        asm volatile("{\n\t.reg .u32 t;\n\tatom.add.acq_rel.gpu.u32 t, [%0], 1;\n}" ::"l"(b.count)
                     : "memory");
    }
}

__device__ bool grid_wait(const BarK& b, unsigned epoch)
{
    __shared__ int s_ok;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const unsigned target = epoch * b.expected;
        int ok = 1;
        const unsigned long long t0 = global_ns();
        // every poll is an L2 round trip (>= 64 ns); the error flag and the
        // clock are checked every 8th poll
        const unsigned long long max_polls = b.timeout_ns / 64ull + 1024ull;
        unsigned long long polls = 0;
        volatile int* verr = b.err;
        for (;;) {
            unsigned cur;
            asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(b.count) : "memory");
            if (cur >= target) break;
            if ((++polls & 7ull) == 0) {
                if (*verr) { ok = 0; break; }
                if (global_ns() - t0 > b.timeout_ns || polls > max_polls) {
                    atomicExch(b.err, 1);
                    ok = 0;
                    break;
                }
            }
        }
        if (ok && *verr) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------- forward: Eq. 2

struct SrcRecK {
    int src_c;            // window state index of the source cell
    float src_scale;      // dt / V
    const float* wavelet; // [nt]
    const int* recmap;    // [nz]: receiver number of cell (0, j) or -1
    float* seis;          // [nrec_max][nt] of this shot
    int nt;
};

struct __align__(16) FwdSmem {
    Tile a, b, c, d;
    Prof pf;
};

// The arithmetic of the velocity half-step of one tile, from the staged
// stresses and the own-node inputs (shared by every kernel that runs it, so
// that they agree bit for bit).
template <int PM>
__device__ __forceinline__ void fwd_vel_core(const WinK& g, const StateK& S, ptrdiff_t fout,
                                             float* hist0,
                                             const Own& o, bool pml, const V4& vr0, const V4& vz0,
                                             const V4& br, const V4& bz, const V4& q0,
                                             const V4& q1, const V4& q2, const V4& q3, float ivr,
                                             float ivh, const Tile& s_rr, const Tile& s_tt,
                                             const Tile& s_rz, const Tile& s_zz, const Prof* pf,
                                             const BarK* bar, unsigned& epoch)
{
    float ari = 0.f, bri = 0.f, arh = 0.f, brh = 0.f;
    V4 azi{}, bzi{}, azh{}, bzh{};
    if (o.live) {
    if (pml) {
        arh = pf->r[0][o.rr];
        brh = pf->r[1][o.rr];
        azh = prof4(pf->z[2], o.cc);
        bzh = prof4(pf->z[3], o.cc);
        if (o.i >= 1) {
            ari = pf->r[2][o.rr];
            bri = pf->r[3][o.rr];
            azi = prof4(pf->z[0], o.cc);
            bzi = prof4(pf->z[1], o.cc);
        }
    }
    const int rr = o.rr, cc = o.cc;
    const V12 rz12 = lds12(s_rz, rr, cc - 4);
    const V4 rzp1 = lds4(s_rz, rr + 1, cc);
    if (o.i >= 1) {
        const V4 rm2 = lds4(s_rr, rr - 2, cc), rm1 = lds4(s_rr, rr - 1, cc);
        const V4 r0 = lds4(s_rr, rr, cc), rp1 = lds4(s_rr, rr + 1, cc);
        const V4 tm1 = lds4(s_tt, rr - 1, cc), t0 = lds4(s_tt, rr, cc);
        const float inv_r = ivr;
        float vr[4], w0[4], w1[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float d_trr = d4(r0.v[e], rm1.v[e], rp1.v[e], rm2.v[e]) * g.inv_dr;
            float d_trz = d4(rz12.v[4 + e], rz12.v[3 + e], rz12.v[5 + e], rz12.v[2 + e]) * g.inv_dz;
            const float hoop = 0.5f * ((rm1.v[e] - tm1.v[e]) + (r0.v[e] - t0.v[e])) * inv_r;
            if (pml) {
                if (ari != 0.f) {
                    w0[e] = bri * q0.v[e] + ari * d_trr;
                    d_trr += w0[e];
                }
                if (azi.v[e] != 0.f) {
                    w1[e] = bzi.v[e] * q1.v[e] + azi.v[e] * d_trz;
                    d_trz += w1[e];
                } else {
                    w1[e] = q1.v[e];  // outside the layer the memory stays 0
                }
            }
            vr[e] = vr0.v[e] + g.dt * br.v[e] * (d_trr + d_trz + hoop);
        }
        st4(S.vr + fout + o.c, o.j, g.nz, vr);
        if (pml) {
            if (ari != 0.f) st4(S.psi_w[0] + o.c, o.j, g.nz, w0);
            st4(S.psi_w[1] + o.c, o.j, g.nz, w1);
        }
    }
    {
        const V12 zz12 = lds12(s_zz, rr, cc - 4);
        const V4 rzm1 = lds4(s_rz, rr - 1, cc), rzp2 = lds4(s_rz, rr + 2, cc);
        const float inv_r = ivh;
        float vz[4], w2[4], w3[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float d_trz = d4(rzp1.v[e], rz12.v[4 + e], rzp2.v[e], rzm1.v[e]) * g.inv_dr;
            float d_tzz = d4(zz12.v[5 + e], zz12.v[4 + e], zz12.v[6 + e], zz12.v[3 + e]) * g.inv_dz;
            const float hoop = 0.5f * (rz12.v[4 + e] + rzp1.v[e]) * inv_r;
            if (pml) {
                if (arh != 0.f) {
                    w2[e] = brh * q2.v[e] + arh * d_trz;
                    d_trz += w2[e];
                }
                if (azh.v[e] != 0.f) {
                    w3[e] = bzh.v[e] * q3.v[e] + azh.v[e] * d_tzz;
                    d_tzz += w3[e];
                } else {
                    w3[e] = q3.v[e];
                }
            }
            vz[e] = vz0.v[e] + g.dt * bz.v[e] * (d_trz + d_tzz + hoop);
        }
        st4(S.vz + fout + o.c, o.j, g.nz, vz);
        if (pml) {
            if (arh != 0.f) st4(S.psi_w[2] + o.c, o.j, g.nz, w2);
            st4(S.psi_w[3] + o.c, o.j, g.nz, w3);
        }
    }
    }
    if (bar) grid_arrive(*bar, epoch);
    if (o.live && hist0) {
        st4(hist0 + o.c, o.j, g.nz, vr0.v);
        st4(hist0 + g.nr * g.P + o.c, o.j, g.nz, vz0.v);
    }
}

// Velocity half-step of one tile: Eq. 2 lines 1-2 with the C-PML memories
// 0..3.  Own-node inputs are loaded before the staging, so the tile pays
// one round trip to L2.  hist0 (or null): history slot receiving v^{n-1/2}.
template <int PM>
__device__ __forceinline__ void fwd_vel_tile(const WinK& g, const CoefK& C, const StateK& S,
                                             ptrdiff_t fin, ptrdiff_t fout, float* hist0, int i0,
                                             int j0, int flags,
                                             const BarK* bar, unsigned& epoch, FwdSmem& sm)
{
    Tile &s_rr = sm.a, &s_tt = sm.b, &s_rz = sm.c, &s_zz = sm.d;
    const Own o = own_of(g, i0, j0);
    const bool pml = tile_pml<PM>(flags);
    V4 vr0{}, vz0{}, br{}, bz{}, q0{}, q1{}, q2{}, q3{};
    float ivr = 0.f, ivh = 0.f;
    __syncthreads();
    for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
        const Slot sl = slot_of(it, i0, j0, g);
        stage_async<EVEN>(s_rr, S.trr + fin, sl);
        stage_async<EVEN>(s_tt, S.ttt + fin, sl);
        stage_async<ODD>(s_rz, S.trz + fin, sl);
        stage_async<EVEN>(s_zz, S.tzz + fin, sl);
    }
    if (pml) stage_prof(sm.pf, C, g, i0, j0);
    // own-node inputs, in flight together with the copies
    if (o.live) {
        ivr = __ldg(C.inv_r_int + o.i);
        ivh = __ldg(C.inv_r_half + o.i);
        vz0 = ld4cg(S.vz + fin + o.c);
        bz = ld4g(C.w_bvz + o.cw);
        if (flags & TILE_LAST) patch4(bz, o.j, g.nz - 1, bvz_at(C, g, o.i, g.nz - 1));
        if (o.i >= 1) {
            vr0 = ld4cg(S.vr + fin + o.c);
            br = ld4g(C.w_bvr + o.cw);
        }
        if (pml) {
            q2 = ld4cg(S.psi[2] + o.c);
            q3 = ld4cg(S.psi[3] + o.c);
            if (o.i >= 1) {
                q0 = ld4cg(S.psi[0] + o.c);
                q1 = ld4cg(S.psi[1] + o.c);
            }
        }
    }
    async_wait_all();
    if (i0 < kH) {
        for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
            const Slot sl = slot_of(it, i0, j0, g);
            if (sl.neg && sl.off_o >= 0) negate_slot(s_rz, sl);
        }
    }
    __syncthreads();
    fwd_vel_core<PM>(g, S, fout, hist0, o, pml, vr0, vz0, br, bz, q0, q1, q2, q3, ivr, ivh, s_rr, s_tt,
                     s_rz, s_zz, &sm.pf, bar, epoch);
}

// The arithmetic of the stress half-step of one tile, from the staged
// velocities and the own-node inputs (shared by every kernel that runs it).
template <int PM>
__device__ __forceinline__ void fwd_stress_core(const WinK& g, const StateK& S, ptrdiff_t fout,
                                                const SrcRecK& q,
                                                int n, bool record, float* hist, const Own& o,
                                                bool pml, const V4& t_rr, const V4& t_tt,
                                                const V4& t_zz, const V4& t_rz, const V4& lm,
                                                const V4& mu, const V4& mh, const V4& q4,
                                                const V4& q5, const V4& q6, const V4& q7,
                                                float ivh, const Tile& s_vr, const Tile& s_vz,
                                                const Prof* pf, const BarK* bar, unsigned& epoch)
{
    const int rr = o.rr, cc = o.cc;
    float arh = 0.f, brh = 0.f;
    V4 azi{}, bzi{};
    if (o.live) {
        if (pml) {
            arh = pf->r[0][rr];
            brh = pf->r[1][rr];
            azi = prof4(pf->z[0], cc);
            bzi = prof4(pf->z[1], cc);
        }
        const V12 vr12 = lds12(s_vr, rr, cc - 4), vz12 = lds12(s_vz, rr, cc - 4);
        const V4 vrp1 = lds4(s_vr, rr + 1, cc);
        const float inv_rh = ivh;
        float trr[4], ttt[4], tzz[4], w4[4], w5[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float d_vr = d4(vrp1.v[e], vr12.v[4 + e], s_vr[rr + 2][cc + e], s_vr[rr - 1][cc + e]) *
                         g.inv_dr;
            const float vr_r = 0.5f * (vr12.v[4 + e] + vrp1.v[e]) * inv_rh;
            float d_vz = d4(vz12.v[4 + e], vz12.v[3 + e], vz12.v[5 + e], vz12.v[2 + e]) * g.inv_dz;
            if (pml) {
                if (arh != 0.f) {
                    w4[e] = brh * q4.v[e] + arh * d_vr;
                    d_vr += w4[e];
                }
                if (azi.v[e] != 0.f) {
                    w5[e] = bzi.v[e] * q5.v[e] + azi.v[e] * d_vz;
                    d_vz += w5[e];
                } else {
                    w5[e] = q5.v[e];
                }
            }
            const float lam = lm.v[e];
            const float l2m = lam + 2.f * mu.v[e];
            trr[e] = t_rr.v[e] + g.dt * (l2m * d_vr + lam * (vr_r + d_vz));
            ttt[e] = t_tt.v[e] + g.dt * (l2m * vr_r + lam * (d_vr + d_vz));
            tzz[e] = t_zz.v[e] + g.dt * (l2m * d_vz + lam * (d_vr + vr_r));
            if (o.c + e == q.src_c) {
                const float inj = q.src_scale * q.wavelet[n];
                trr[e] += inj;
                ttt[e] += inj;
                tzz[e] += inj;
            }
            if (o.i == 0 && record && o.j + e < g.nz) {
                const int k = q.recmap[o.j + e];
                if (k >= 0) q.seis[(size_t)k * q.nt + n] = (trr[e] + ttt[e] + tzz[e]) * (1.f / 3.f);
            }
        }
        st4(S.trr + fout + o.c, o.j, g.nz, trr);
        st4(S.ttt + fout + o.c, o.j, g.nz, ttt);
        st4(S.tzz + fout + o.c, o.j, g.nz, tzz);
        if (pml) {
            if (arh != 0.f) st4(S.psi_w[4] + o.c, o.j, g.nz, w4);
            st4(S.psi_w[5] + o.c, o.j, g.nz, w5);
        }
    }
    if (o.live && o.i >= 1) {
        float ari = 0.f, bri = 0.f;
        V4 azh{}, bzh{};
        if (pml) {
            ari = pf->r[2][rr];
            bri = pf->r[3][rr];
            azh = prof4(pf->z[2], cc);
            bzh = prof4(pf->z[3], cc);
        }
        const V12 vr12 = lds12(s_vr, rr, cc - 4);
        const V4 vz0 = lds4(s_vz, rr, cc), vzm1 = lds4(s_vz, rr - 1, cc),
                 vzm2 = lds4(s_vz, rr - 2, cc), vzp1 = lds4(s_vz, rr + 1, cc);
        float trz[4], w6[4], w7[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float d_vrz = d4(vr12.v[5 + e], vr12.v[4 + e], vr12.v[6 + e], vr12.v[3 + e]) * g.inv_dz;
            float d_vzr = d4(vz0.v[e], vzm1.v[e], vzp1.v[e], vzm2.v[e]) * g.inv_dr;
            if (pml) {
                if (azh.v[e] != 0.f) {
                    w6[e] = bzh.v[e] * q6.v[e] + azh.v[e] * d_vrz;
                    d_vrz += w6[e];
                } else {
                    w6[e] = q6.v[e];
                }
                if (ari != 0.f) {
                    w7[e] = bri * q7.v[e] + ari * d_vzr;
                    d_vzr += w7[e];
                }
            }
            trz[e] = t_rz.v[e] + g.dt * mh.v[e] * (d_vrz + d_vzr);
        }
        st4(S.trz + fout + o.c, o.j, g.nz, trz);
        if (pml) {
            st4(S.psi_w[6] + o.c, o.j, g.nz, w6);
            if (ari != 0.f) st4(S.psi_w[7] + o.c, o.j, g.nz, w7);
        }
    }
    // the history is read only by the adjoint, after this launch
    if (bar) grid_arrive(*bar, epoch);
    if (o.live && hist) {
        const V4 a = lds4(s_vr, rr, cc), b = lds4(s_vz, rr, cc);
        st4(hist + o.c, o.j, g.nz, a.v);
        st4(hist + g.nr * g.P + o.c, o.j, g.nz, b.v);
    }
}

// Stress half-step of one tile: Eq. 2 lines 3-6 with the C-PML memories
// 4..7, source injection into the three normal stresses, pressure
// recording, and the store of v^{n+1/2} for the adjoint.
template <int PM>
__device__ __forceinline__ void fwd_stress_tile(const WinK& g, const CoefK& C, const StateK& S,
                                                ptrdiff_t fin, ptrdiff_t fout, const SrcRecK& q,
                                                int n, bool record,
                                                float* hist, int i0, int j0, int flags,
                                                const BarK* bar, unsigned& epoch, FwdSmem& sm)
{
    Tile &s_vr = sm.a, &s_vz = sm.b;
    const Own o = own_of(g, i0, j0);
    const bool pml = tile_pml<PM>(flags);
    __syncthreads();
    for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
        const Slot sl = slot_of(it, i0, j0, g);
        stage_async<ODD>(s_vr, S.vr + fout, sl);
        stage_async<EVEN>(s_vz, S.vz + fout, sl);
    }
    if (pml) stage_prof(sm.pf, C, g, i0, j0);
    V4 t_rr{}, t_tt{}, t_zz{}, lm{}, mu{}, t_rz{}, mh{};
    float ivh = 0.f;
    V4 q4{}, q5{}, q6{}, q7{};
    if (o.live) {
        ivh = __ldg(C.inv_r_half + o.i);
        t_rr = ld4cg(S.trr + fin + o.c);
        t_tt = ld4cg(S.ttt + fin + o.c);
        t_zz = ld4cg(S.tzz + fin + o.c);
        lm = ld4g(C.w_lam + o.cw);
        mu = ld4g(C.w_mu + o.cw);
        if (o.i >= 1) {
            t_rz = ld4cg(S.trz + fin + o.c);
            mh = ld4g(C.w_muh + o.cw);
            if (flags & TILE_LAST) patch4(mh, o.j, g.nz - 1, muh_at(C, g, o.i, g.nz - 1));
        }
        if (pml) {
            q4 = ld4cg(S.psi[4] + o.c);
            q5 = ld4cg(S.psi[5] + o.c);
            if (o.i >= 1) {
                q6 = ld4cg(S.psi[6] + o.c);
                q7 = ld4cg(S.psi[7] + o.c);
            }
        }
    }
    async_wait_all();
    if (i0 < kH) {
        for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
            const Slot sl = slot_of(it, i0, j0, g);
            if (sl.neg && sl.off_o >= 0) negate_slot(s_vr, sl);
        }
    }
    __syncthreads();
    fwd_stress_core<PM>(g, S, fout, q, n, record, hist, o, pml, t_rr, t_tt, t_zz, t_rz, lm, mu, mh, q4,
                        q5, q6, q7, ivh, s_vr, s_vz, &sm.pf, bar, epoch);
}

// ------------------------------------------ adjoint: transpose of Eq. 2
//
// Gather form of the transpose.  The forward step reads ghost values through
// the axis mirror and the zero edges; the transpose of "mirror, then
// stencil" is "stencil of the coefficients extended with the same parity,
// then fold", which here means: the transposed stencil reads the adjoint
// coefficients of cells and v_z nodes with the even extension
// (X[-1-k] = X[k]), those of v_r and trz nodes with the odd extension
// (X[-k] = -X[k], X[0] = 0), and zero beyond the edges.

struct AdjK {
    const float* resid;   // [nrec_max][nt] of this shot
    const int* recmap;    // [nz]
    int nt;
    float2 *G_lam, *G_munn, *G_murz, *G_br, *G_bz;  // Kahan pairs [nr*P]
    float *H_lam, *H_munn, *H_murz;                 // [nr*P]
};

struct __align__(16) AdjSmem {
    // d: tiles of both half-steps.  Stress step: adjoint stresses (d0..d3),
    // adjoint memories 4..7 (d4..d7; d6, d7 then hold the coefficients on
    // D_z v_r and D_r v_z at shear nodes).  Velocity step: adjoint
    // velocities (d0, d1), memories 0..3 (d2..d5), buoyancies (d6, d7), each
    // replaced in place by W = dt b Av and the four coefficients.
    // f: stress step only, data that do not change within a launch: forward
    // v_r, v_z of v^{n+1/2} (f0, f1) and lambda, mu, mu_h (f2..f4, replaced
    // in place by the coefficients on D_r v_r, v_r/r and D_z v_z at cells).
    // The velocity step of reverse step n stages f for step n-1 once its
    // own tiles are built, so those copies run during the grid barrier.
    Tile d[8];
    Tile f[5];
    Prof pf;
};

// Shared memory of launches that cover one tile class only.  Interior
// tiles stage no C-PML memories and their shear coefficient tiles x6, x7
// hold equal values, so the stress step needs 10 tiles (6 blocks per SM
// instead of 5); the velocity step keeps W, the coefficients (equal to W on
// interior tiles) and the buoyancies: 8 tiles, or 4 on interior tiles.
struct __align__(16) AdjStressIntSmem {
    Tile d[5];
    Tile f[5];
    Prof pf;
};

template <int K>
struct __align__(16) AdjVelSmem {
    Tile d[K];
    Prof pf;
};

// the stress step's launch-invariant tiles (see AdjSmem)
template <typename SM>
__device__ __forceinline__ void stage_adj_statics(SM& sm, const CoefK& C, const float* fcur,
                                                  int i0, int j0, const WinK& g)
{
    const int plane = g.nr * g.P;
    for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
        const Slot sl = slot_of(it, i0, j0, g);
        stage_async<ODD>(sm.f[0], fcur, sl);
        stage_async<EVEN>(sm.f[1], fcur + plane, sl);
        stage_async<EVEN, true>(sm.f[2], C.w_lam, sl);
        stage_async<EVEN, true>(sm.f[3], C.w_mu, sl);
        stage_async<ABS, true>(sm.f[4], C.w_muh, sl);
    }
}

__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// The tile's own accumulator lines (Kahan pairs, pseudo-Hessian; with RHO
// also the density pairs and v^{n-1/2}) are read only at the end of the
// stress step: ask for them in L2 while the tile is staged.  Rows of 32
// nodes start 128-byte aligned (P and j0 are multiples of 32); only rows
// inside the window are touched.
template <bool RHO>
__device__ __forceinline__ void prefetch_accumulators(const WinK& g, const AdjK& q,
                                                      const float* fprev, int i0, int j0)
{
    constexpr int kLines = RHO ? 14 : 9;  // 128-byte lines per tile row
    for (int k = tid_of(); k < kTR * kLines; k += kThreads) {
        const int row = k / kLines, l = k - row * kLines;
        const int i = i0 + row;
        if (i >= g.nr) continue;
        const size_t c = (size_t)i * g.P + j0;
        const char* p;
        switch (l) {
        case 0: case 1: p = (const char*)(q.G_lam + c) + 128 * l; break;
        case 2: case 3: p = (const char*)(q.G_munn + c) + 128 * (l - 2); break;
        case 4: case 5: p = (const char*)(q.G_murz + c) + 128 * (l - 4); break;
        case 6: p = (const char*)(q.H_lam + c); break;
        case 7: p = (const char*)(q.H_munn + c); break;
        case 8: p = (const char*)(q.H_murz + c); break;
        case 9: case 10: p = (const char*)(q.G_br + c) + 128 * (l - 9); break;
        case 11: case 12: p = (const char*)(q.G_bz + c) + 128 * (l - 11); break;
        default: p = (const char*)(fprev + c); break;
        }
        prefetch_l2(p);
    }
}

__device__ __forceinline__ float2 kahan_step(float2 s, float x)
{
    float y = __fsub_rn(x, s.y);
    float t = __fadd_rn(s.x, y);
    s.y = __fsub_rn(__fsub_rn(t, s.x), y);
    s.x = t;
    return s;
}

// Transpose of the stress step of one tile at reverse step n, fused with
// the gradient correlations (Eq. 7, Eq. 8, and the density term).
// S.{trr..trz} hold dJ/dtau^{n+1}; S.{vr,vz} accumulate to dJ/dv^{n+1/2};
// psi[4..7] are the adjoint memories read side, psi_w[4..7] the write side.
// fcur: v_r, v_z planes of v^{n+1/2}; fprev: those of v^{n-1/2}.
// Shear-mu correlation (Eq. 8), the shear pseudo-Hessian and, with RHO,
// the density correlation at one tile's own nodes for reverse step n, from
// the staged forward velocities v^{n+1/2} (fr, fz), v^{n-1/2} (fprev, read
// only with RHO), the own adjoint velocities Av^{n+1/2} and the own adjoint
// trz of step n+1.  Without RHO (the caller asks for no density gradient)
// neither v^{n-1/2} nor the density accumulators are touched.
template <bool RHO>
__device__ __forceinline__ void adj_corr_shear(const WinK& g, const AdjK& q, const Own& o,
                                               const float* fprev, const Tile& T_fr,
                                               const Tile& T_fz, const V4& Arz,
                                               const float (&avz)[4], const float (&avr)[4])
{
    const int plane = g.nr * g.P, c = o.c, rr = o.rr, cc = o.cc, i = o.i;
    const float dt = g.dt;
    float2 gbz[4], gmr[4], gbr[4];
    V4 pz{}, hmr{}, pr{};
    if (RHO) {
        ld4f2(q.G_bz + c, gbz);
        pz = ld4cg(fprev + plane + c);
    }
    if (i >= 1) {
        ld4f2(q.G_murz + c, gmr);
        hmr = ld4cg(q.H_murz + c);
        if (RHO) {
            pr = ld4cg(fprev + c);
            ld4f2(q.G_br + c, gbr);
        }
    }
    const V4 fz0 = lds4(T_fz, rr, cc);
    if (RHO) {
#pragma unroll
        for (int e = 0; e < 4; ++e) gbz[e] = kahan_step(gbz[e], (fz0.v[e] - pz.v[e]) * avz[e]);
        st4f2(q.G_bz + c, o.j, g.nz, gbz);
    }
    if (i >= 1) {
        const V12 fr12 = lds12(T_fr, rr, cc - 4);
        const V4 fzm1 = lds4(T_fz, rr - 1, cc), fzm2 = lds4(T_fz, rr - 2, cc),
                 fzp1 = lds4(T_fz, rr + 1, cc);
        float hmr2[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float gam =
                d4(fr12.v[5 + e], fr12.v[4 + e], fr12.v[6 + e], fr12.v[3 + e]) * g.inv_dz +
                d4(fz0.v[e], fzm1.v[e], fzp1.v[e], fzm2.v[e]) * g.inv_dr;
            gmr[e] = kahan_step(gmr[e], dt * gam * Arz.v[e]);
            hmr2[e] = hmr.v[e] + dt * gam * gam;
            if (RHO) gbr[e] = kahan_step(gbr[e], (fr12.v[4 + e] - pr.v[e]) * avr[e]);
        }
        st4f2(q.G_murz + c, o.j, g.nz, gmr);
        st4(q.H_murz + c, o.j, g.nz, hmr2);
        if (RHO) st4f2(q.G_br + c, o.j, g.nz, gbr);
    }
}

// statics: the f tiles were staged by the preceding velocity step.
// defer: adj_corr_shear runs in the velocity step of the same reverse step
// (the block keeps this tile, so the f tiles are still in shared memory).
// bar (or null): the block arrives at the grid barrier once the adjoint
// velocities are stored; the own-node correlations follow the arrival.
template <bool RHO, int PM, typename SM>
__device__ __forceinline__ void adj_stress_tile(const WinK& g, const CoefK& C, const StateK& S,
                                                const AdjK& q, const float* fcur,
                                                const float* fprev, int i0, int j0, int flags,
                                                bool statics, bool defer, const BarK* bar,
                                                unsigned& epoch, SM& sm)
{
    const float dt = g.dt;
    const Own o = own_of(g, i0, j0);
    const bool pml = tile_pml<PM>(flags);
    const int rr = o.rr, cc = o.cc, i = o.i, c = o.c;
    // interior tiles stage no C-PML memories, and their x6 and x7 are equal
    constexpr bool kInt = PM == PM_INTERIOR;
    Tile &T_rr = sm.d[0], &T_tt = sm.d[1], &T_zz = sm.d[2], &T_rz = sm.d[3];
    Tile &T_p4 = sm.d[kInt ? 0 : 4], &T_p5 = sm.d[kInt ? 0 : 5], &T_x6 = sm.d[kInt ? 4 : 6],
         &T_x7 = sm.d[kInt ? 4 : 7];
    Tile &T_fr = sm.f[0], &T_fz = sm.f[1], &T_x4 = sm.f[2], &T_yt = sm.f[3], &T_x5 = sm.f[4];
    __syncthreads();
    if (!statics) stage_adj_statics(sm, C, fcur, i0, j0, g);
    for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
        const Slot sl = slot_of(it, i0, j0, g);
        stage_async<EVEN>(T_rr, S.trr, sl);
        stage_async<EVEN>(T_tt, S.ttt, sl);
        stage_async<EVEN>(T_zz, S.tzz, sl);
        stage_async<ODD>(T_rz, S.trz, sl);
        if (pml) {
            stage_async<EVEN>(T_p4, S.psi[4], sl);
            stage_async<EVEN>(T_p5, S.psi[5], sl);
            stage_async<POS>(T_x6, S.psi[6], sl);
            stage_async<POS>(T_x7, S.psi[7], sl);
        }
    }
    if (pml) stage_prof(sm.pf, C, g, i0, j0);
    prefetch_accumulators<RHO>(g, q, fprev, i0, j0);
    // own adjoint velocities, in flight together with the copies
    V4 av_z{}, av_r{};
    float ivh = 0.f, ivm = 0.f;
    if (o.live) {
        av_z = ld4cg(S.vz + c);
        ivh = __ldg(C.inv_r_half + i);
        if (i >= 1) {
            av_r = ld4cg(S.vr + c);
            ivm = __ldg(C.inv_r_half + i - 1);
        }
    }
    async_wait_all();
    if (i0 < kH) {
        for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
            const Slot sl = slot_of(it, i0, j0, g);
            if (sl.neg && sl.off_o >= 0) {
                negate_slot(T_rz, sl);
                negate_slot(T_fr, sl);
            }
        }
    }
    __syncthreads();

    // transposed-stencil coefficients, in place over this thread's slots;
    // own C-PML nodes also update their adjoint memories here
    for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
        const Slot sl = slot_of(it, i0, j0, g);
        const int r2 = sl.rr, c2 = sl.cq;
        const int ii = i0 - kH + r2, j = j0 - 4 + c2;
        const V4 lm = lds4(T_x4, r2, c2), mu = lds4(T_yt, r2, c2);
        V4 mh = lds4(T_x5, r2, c2);
        if ((flags & TILE_LAST) && sl.offw_o >= 0) {
            // the window's last trz row (the copy holds the global model's)
            const int io = ii < 0 ? -ii : ii;
            patch4(mh, j, g.nz - 1, muh_at(C, g, io, g.nz - 1));
        }
        const V4 ar = lds4(T_rr, r2, c2), at = lds4(T_tt, r2, c2), az = lds4(T_zz, r2, c2);
        const V4 arz = lds4(T_rz, r2, c2);
        float x4[4], ytt[4], x5[4], x6[4], x7[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float lam = lm.v[e], l2m = lam + 2.f * mu.v[e];
            x4[e] = dt * (l2m * ar.v[e] + lam * (at.v[e] + az.v[e]));
            ytt[e] = dt * (l2m * at.v[e] + lam * (ar.v[e] + az.v[e]));
            x5[e] = dt * (l2m * az.v[e] + lam * (ar.v[e] + at.v[e]));
            // shear node: the staged values are already odd about the axis
            x6[e] = x7[e] = dt * mh.v[e] * arz.v[e];
        }
        if (pml && ii < g.nr && j >= 0 && j < g.nz) {
            const bool own = own_slot(sl);
            const float arh = sm.pf.r[0][r2], brh = sm.pf.r[1][r2];
            const V4 p4 = lds4(T_p4, r2, c2), p5 = lds4(T_p5, r2, c2);
            const V4 azi = prof4(sm.pf.z[0], c2), bzi = prof4(sm.pf.z[1], c2);
            if (own) {
                float w4[4], w5[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    w4[e] = x4[e] + brh * p4.v[e];
                    w5[e] = x5[e] + bzi.v[e] * p5.v[e];
                }
                if (arh != 0.f) st4(S.psi_w[4] + ii * g.P + j, j, g.nz, w4);
                st4(S.psi_w[5] + ii * g.P + j, j, g.nz, w5);
            }
            if (arh != 0.f) {
#pragma unroll
                for (int e = 0; e < 4; ++e) x4[e] = x4[e] + arh * (x4[e] + brh * p4.v[e]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (azi.v[e] != 0.f) x5[e] = x5[e] + azi.v[e] * (x5[e] + bzi.v[e] * p5.v[e]);
            if (ii >= 1) {
                const V4 azh = prof4(sm.pf.z[2], c2), bzh = prof4(sm.pf.z[3], c2);
                const float ari = sm.pf.r[2][r2], bri = sm.pf.r[3][r2];
                const V4 p6 = lds4(T_x6, r2, c2), p7 = lds4(T_x7, r2, c2);
                if (own) {
                    float w6[4], w7[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        w6[e] = x6[e] + bzh.v[e] * p6.v[e];
                        w7[e] = x7[e] + bri * p7.v[e];
                    }
                    st4(S.psi_w[6] + ii * g.P + j, j, g.nz, w6);
                    if (ari != 0.f) st4(S.psi_w[7] + ii * g.P + j, j, g.nz, w7);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (azh.v[e] != 0.f) x6[e] = x6[e] + azh.v[e] * (x6[e] + bzh.v[e] * p6.v[e]);
                if (ari != 0.f) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) x7[e] = x7[e] + ari * (x7[e] + bri * p7.v[e]);
                }
            }
        }
        *reinterpret_cast<float4*>(&T_x4[r2][c2]) = make_float4(x4[0], x4[1], x4[2], x4[3]);
        *reinterpret_cast<float4*>(&T_yt[r2][c2]) = make_float4(ytt[0], ytt[1], ytt[2], ytt[3]);
        *reinterpret_cast<float4*>(&T_x5[r2][c2]) = make_float4(x5[0], x5[1], x5[2], x5[3]);
        *reinterpret_cast<float4*>(&T_x6[r2][c2]) = make_float4(x6[0], x6[1], x6[2], x6[3]);
        *reinterpret_cast<float4*>(&T_x7[r2][c2]) = make_float4(x7[0], x7[1], x7[2], x7[3]);
    }
    __syncthreads();

    // ---- transpose of the stress step into Av
    float avz[4] = {0.f, 0.f, 0.f, 0.f}, avr[4] = {0.f, 0.f, 0.f, 0.f};
    if (o.live) {
        const V12 x5r = lds12(T_x5, rr, cc - 4);
        const V4 x7m1 = lds4(T_x7, rr - 1, cc), x70 = lds4(T_x7, rr, cc),
                 x7p1 = lds4(T_x7, rr + 1, cc), x7p2 = lds4(T_x7, rr + 2, cc);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float s = d4(x5r.v[4 + e], x5r.v[5 + e], x5r.v[3 + e], x5r.v[6 + e]) * g.inv_dz;
            s += d4(x70.v[e], x7p1.v[e], x7m1.v[e], x7p2.v[e]) * g.inv_dr;
            avz[e] = av_z.v[e] + s;
        }
        st4(S.vz + c, o.j, g.nz, avz);
        if (i >= 1) {
            const V4 x4m2 = lds4(T_x4, rr - 2, cc), x4m1 = lds4(T_x4, rr - 1, cc),
                     x40 = lds4(T_x4, rr, cc), x4p1 = lds4(T_x4, rr + 1, cc);
            const V4 ytm1 = lds4(T_yt, rr - 1, cc), yt0 = lds4(T_yt, rr, cc);
            const V12 x6r = lds12(T_x6, rr, cc - 4);
            const float irm = ivm, inv_rh = ivh;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float s = d4(x4m1.v[e], x40.v[e], x4m2.v[e], x4p1.v[e]) * g.inv_dr;
                s += 0.5f * (ytm1.v[e] * irm + yt0.v[e] * inv_rh);
                s += d4(x6r.v[3 + e], x6r.v[4 + e], x6r.v[2 + e], x6r.v[5 + e]) * g.inv_dz;
                avr[e] = av_r.v[e] + s;
            }
            st4(S.vr + c, o.j, g.nz, avr);
        }
    }
    // everything the next phase reads from this tile is stored
    if (bar) grid_arrive(*bar, epoch);
    if (!o.live) return;

    // ---- lambda and normal-mu correlations (Eq. 7, Eq. 8) and pseudo-Hessian
    float2 gl[4], gm[4];
    ld4f2(q.G_lam + c, gl);
    ld4f2(q.G_munn + c, gm);
    const V4 hl = ld4cg(q.H_lam + c), hm = ld4cg(q.H_munn + c);
    float hl2[4], hm2[4];
    {
        const V12 fr12 = lds12(T_fr, rr, cc - 4), fz12 = lds12(T_fz, rr, cc - 4);
        const V4 frm1 = lds4(T_fr, rr - 1, cc), frp1 = lds4(T_fr, rr + 1, cc),
                 frp2 = lds4(T_fr, rr + 2, cc);
        const V4 Arr = lds4(T_rr, rr, cc), Att = lds4(T_tt, rr, cc), Azz = lds4(T_zz, rr, cc);
        const float inv_rh = ivh;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float err = d4(frp1.v[e], fr12.v[4 + e], frp2.v[e], frm1.v[e]) * g.inv_dr;
            const float ett = 0.5f * (fr12.v[4 + e] + frp1.v[e]) * inv_rh;
            const float ezz = d4(fz12.v[4 + e], fz12.v[3 + e], fz12.v[5 + e], fz12.v[2 + e]) * g.inv_dz;
            const float div = err + ett + ezz;
            gl[e] = kahan_step(gl[e], dt * div * (Arr.v[e] + Att.v[e] + Azz.v[e]));
            gm[e] = kahan_step(gm[e], 2.f * dt * (err * Arr.v[e] + ett * Att.v[e] + ezz * Azz.v[e]));
            hl2[e] = hl.v[e] + dt * div * div;
            hm2[e] = hm.v[e] + 4.f * dt * (err * err + ett * ett + ezz * ezz);
        }
    }
    st4f2(q.G_lam + c, o.j, g.nz, gl);
    st4f2(q.G_munn + c, o.j, g.nz, gm);
    st4(q.H_lam + c, o.j, g.nz, hl2);
    st4(q.H_munn + c, o.j, g.nz, hm2);
    if (!defer) adj_corr_shear<RHO>(g, q, o, fprev, T_fr, T_fz, lds4(T_rz, rr, cc), avz, avr);
}

// Transpose of the velocity step of one tile at reverse step n: S.{vr,vz}
// hold dJ/dv^{n+1/2}; S.{trr..trz} accumulate to dJ/dtau^n.  Then the
// residual of step n-1 is injected at the receivers (transpose of the
// recording).
// next_fcur (or null): v^{n-1/2}, whose stress step (reverse step n-1) runs
// next on this tile; its launch-invariant tiles are staged here, after the
// block's arrival at the grid barrier (bar, or null: no barrier), and after
// the correlations deferred by the stress step (fprev_b, or null).
template <bool RHO, int PM, bool PERSIST, typename SM>
__device__ __forceinline__ void adj_vel_tile(const WinK& g, const CoefK& C, const StateK& S,
                                             const AdjK& q, int n, int i0, int j0, int flags,
                                             const float* next_fcur, const float* fprev_b,
                                             const BarK* bar, unsigned& epoch, SM& sm)
{
    // W = dt b Av at the velocity nodes (odd about the axis for v_r, even
    // for v_z) and the coefficients on the four stretched derivatives; on
    // interior tiles the coefficients are W itself and share its tiles
    constexpr bool kInt = PM == PM_INTERIOR;
    Tile &s_wr = sm.d[0], &s_wz = sm.d[1];
    Tile &s_x0 = sm.d[kInt ? 0 : 2], &s_x1 = sm.d[kInt ? 0 : 3], &s_x2 = sm.d[kInt ? 1 : 4],
         &s_x3 = sm.d[kInt ? 1 : 5], &s_br = sm.d[kInt ? 2 : 6], &s_bz = sm.d[kInt ? 3 : 7];
    const Own o = own_of(g, i0, j0);
    const bool pml = tile_pml<PM>(flags);
    __syncthreads();
    for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
        const Slot sl = slot_of(it, i0, j0, g);
        stage_async<ODD>(s_wr, S.vr, sl);
        stage_async<ABS, true>(s_br, C.w_bvr, sl);
        stage_async<EVEN>(s_wz, S.vz, sl);
        stage_async<EVEN, true>(s_bz, C.w_bvz, sl);
        if (pml) {
            stage_async<ODD>(s_x0, S.psi[0], sl);
            stage_async<ODD>(s_x1, S.psi[1], sl);
            stage_async<EVEN>(s_x2, S.psi[2], sl);
            stage_async<EVEN>(s_x3, S.psi[3], sl);
        }
    }
    if (pml) stage_prof(sm.pf, C, g, i0, j0);
    V4 o_rr{}, o_tt{}, o_zz{}, o_rz{}, r3{};
    float ir0 = 0.f, ir1 = 0.f, irm = 0.f, irh = 0.f;
    if (o.live) {
        ir0 = __ldg(C.inv_r_int + o.i);
        irh = __ldg(C.inv_r_half + o.i);
        if (o.i + 1 < g.nr) ir1 = __ldg(C.inv_r_int + o.i + 1);
        if (o.i >= 1) irm = __ldg(C.inv_r_half + o.i - 1);
        o_rr = ld4cg(S.trr + o.c);
        o_tt = ld4cg(S.ttt + o.c);
        o_zz = ld4cg(S.tzz + o.c);
        if (o.i >= 1) o_rz = ld4cg(S.trz + o.c);
        if (o.i == 0 && n > 0) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = o.j + e < g.nz ? q.recmap[o.j + e] : -1;
                if (k >= 0) r3.v[e] = q.resid[(size_t)k * q.nt + (n - 1)] * (1.f / 3.f);
            }
        }
    }
    async_wait_all();
    if (pml) __syncthreads();  // the profiles come from other threads
    // in place over this thread's slots (read by other threads only after
    // the barrier below); own C-PML nodes also update their adjoint memories
    for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
        const Slot sl = slot_of(it, i0, j0, g);
        const int r2 = sl.rr, c2 = sl.cq;
        const int ii = i0 - kH + r2, j = j0 - 4 + c2;
        const bool own = own_slot(sl);
        if (sl.neg && sl.off_o >= 0) {
            negate_slot(s_wr, sl);
            if (pml) {
                negate_slot(s_x0, sl);
                negate_slot(s_x1, sl);
            }
        }
        // v_r node (zero-filled where there is none)
        {
            const V4 av = lds4(s_wr, r2, c2), bv = lds4(s_br, r2, c2);
            float w[4], x0[4], x1[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) x0[e] = x1[e] = w[e] = g.dt * bv.v[e] * av.v[e];
            if (pml && sl.off_o >= 0) {
                const float ari = sm.pf.r[2][r2], bri = sm.pf.r[3][r2];
                const V4 p0 = lds4(s_x0, r2, c2), p1 = lds4(s_x1, r2, c2);
                const V4 azi = prof4(sm.pf.z[0], c2), bzi = prof4(sm.pf.z[1], c2);
                if (own) {
                    float w0[4], w1[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        w0[e] = w[e] + bri * p0.v[e];
                        w1[e] = w[e] + bzi.v[e] * p1.v[e];
                    }
                    if (ari != 0.f) st4(S.psi_w[0] + ii * g.P + j, j, g.nz, w0);
                    st4(S.psi_w[1] + ii * g.P + j, j, g.nz, w1);
                }
                if (ari != 0.f) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) x0[e] = w[e] + ari * (w[e] + bri * p0.v[e]);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (azi.v[e] != 0.f) x1[e] = w[e] + azi.v[e] * (w[e] + bzi.v[e] * p1.v[e]);
            }
            *reinterpret_cast<float4*>(&s_wr[r2][c2]) = make_float4(w[0], w[1], w[2], w[3]);
            if (!kInt) {
                *reinterpret_cast<float4*>(&s_x0[r2][c2]) = make_float4(x0[0], x0[1], x0[2], x0[3]);
                *reinterpret_cast<float4*>(&s_x1[r2][c2]) = make_float4(x1[0], x1[1], x1[2], x1[3]);
            }
        }
        // v_z node
        {
            const V4 av = lds4(s_wz, r2, c2);
            V4 bv = lds4(s_bz, r2, c2);
            if ((flags & TILE_LAST) && sl.offw_e >= 0) {
                // the window's last v_z row (the copy holds the global model's)
                const int ie = ii < 0 ? -1 - ii : ii;
                patch4(bv, j, g.nz - 1, bvz_at(C, g, ie, g.nz - 1));
            }
            float w[4], x2[4], x3[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) x2[e] = x3[e] = w[e] = g.dt * bv.v[e] * av.v[e];
            if (pml && sl.off_e >= 0) {
                const float arh = sm.pf.r[0][r2], brh = sm.pf.r[1][r2];
                const V4 p2 = lds4(s_x2, r2, c2), p3 = lds4(s_x3, r2, c2);
                const V4 azh = prof4(sm.pf.z[2], c2), bzh = prof4(sm.pf.z[3], c2);
                if (own) {
                    float w2[4], w3[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        w2[e] = w[e] + brh * p2.v[e];
                        w3[e] = w[e] + bzh.v[e] * p3.v[e];
                    }
                    if (arh != 0.f) st4(S.psi_w[2] + ii * g.P + j, j, g.nz, w2);
                    st4(S.psi_w[3] + ii * g.P + j, j, g.nz, w3);
                }
                if (arh != 0.f) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) x2[e] = w[e] + arh * (w[e] + brh * p2.v[e]);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (azh.v[e] != 0.f) x3[e] = w[e] + azh.v[e] * (w[e] + bzh.v[e] * p3.v[e]);
            }
            *reinterpret_cast<float4*>(&s_wz[r2][c2]) = make_float4(w[0], w[1], w[2], w[3]);
            if (!kInt) {
                *reinterpret_cast<float4*>(&s_x2[r2][c2]) = make_float4(x2[0], x2[1], x2[2], x2[3]);
                *reinterpret_cast<float4*>(&s_x3[r2][c2]) = make_float4(x3[0], x3[1], x3[2], x3[3]);
            }
        }
    }
    __syncthreads();
    const int rr = o.rr, cc = o.cc, i = o.i, c = o.c;
    if (o.live) {
        const V4 wr0 = lds4(s_wr, rr, cc), wrp1 = lds4(s_wr, rr + 1, cc);
        const V4 x0m1 = lds4(s_x0, rr - 1, cc), x00 = lds4(s_x0, rr, cc),
                 x0p1 = lds4(s_x0, rr + 1, cc), x0p2 = lds4(s_x0, rr + 2, cc);
        const V12 x3r = lds12(s_x3, rr, cc - 4);
        float trr[4], ttt[4], tzz[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            // cell (i,j); inv_r_int[0] is 0 and W_r vanishes on the axis
            const float hoop = 0.5f * (wr0.v[e] * ir0 + wrp1.v[e] * ir1);
            const float arr = d4(x00.v[e], x0p1.v[e], x0m1.v[e], x0p2.v[e]) * g.inv_dr;
            const float azz = d4(x3r.v[3 + e], x3r.v[4 + e], x3r.v[2 + e], x3r.v[5 + e]) * g.inv_dz;
            trr[e] = o_rr.v[e] + arr + hoop + r3.v[e];
            ttt[e] = o_tt.v[e] - hoop + r3.v[e];
            tzz[e] = o_zz.v[e] + azz + r3.v[e];
        }
        st4(S.trr + c, o.j, g.nz, trr);
        st4(S.ttt + c, o.j, g.nz, ttt);
        st4(S.tzz + c, o.j, g.nz, tzz);
    }
    if (o.live && i >= 1) {
        const V12 x1r = lds12(s_x1, rr, cc - 4);
        const V4 x2m2 = lds4(s_x2, rr - 2, cc), x2m1 = lds4(s_x2, rr - 1, cc),
                 x20 = lds4(s_x2, rr, cc), x2p1 = lds4(s_x2, rr + 1, cc);
        const V4 wzm1 = lds4(s_wz, rr - 1, cc), wz0 = lds4(s_wz, rr, cc);
        float trz[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float s = d4(x1r.v[4 + e], x1r.v[5 + e], x1r.v[3 + e], x1r.v[6 + e]) * g.inv_dz;
            s += d4(x2m1.v[e], x20.v[e], x2m2.v[e], x2p1.v[e]) * g.inv_dr;
            s += 0.5f * (wzm1.v[e] * irm + wz0.v[e] * irh);
            trz[e] = o_rz.v[e] + s;
        }
        st4(S.trz + c, o.j, g.nz, trz);
    }
    if (bar) grid_arrive(*bar, epoch);
    if constexpr (PERSIST) {
        // fprev_b (or null): v^{n-1/2}; the stress step deferred its density
        // and shear correlations to here (own nodes only: no other block
        // reads them)
        if (fprev_b) {
            if (o.live) {
                const V4 az = ld4cg(S.vz + c);
                V4 ar{};
                if (i >= 1) ar = ld4cg(S.vr + c);
                adj_corr_shear<RHO>(g, q, o, fprev_b, sm.f[0], sm.f[1], o_rz, az.v, ar.v);
            }
            __syncthreads();  // the f tiles are read above and refilled below
        }
        // the next stress step's launch-invariant tiles: the copies run during
        // the grid barrier
        if (next_fcur) stage_adj_statics(sm, C, next_fcur, i0, j0, g);
    }
}

// ------------------------------------------------ shots, tiles, runs
//
// Every shot has its own window state; all shots of a model advance in
// lockstep.  One tile table lists (shot, i0, j0) for every tile of every
// shot, so one launch (or one persistent phase) covers all shots.

struct ShotK {
    WinK g;
    CoefK C;
    StateK Sf;      // forward view: C-PML memories updated in place (bank a)
    StateK Sa[2];   // adjoint views: read bank a / write bank b, and reverse
    SrcRecK q;
    AdjK a;
    float* hist;    // history window: slot k = v_r, v_z planes of v^{hist_n0 + k - 1/2}
    // second forward field buffer (fused steps): field f of buffer 1 is
    // Sf.f + swap; the C-PML memories exist once
    long long swap;
};

// The shots of one launch travel in the kernel's parameter space (constant
// bank, no loads in the tile code); batches larger than kGroup run as
// several launches.
constexpr int kGroup = 32;
template <int N>
struct ShotTable {
    ShotK s[N];
};

struct RunK {
    const int4* tiles;  // (shot within the table, i0, j0, TILE_* flags)
    int ntiles;
    int n0, n1;         // forward: steps n0 .. n1-1; adjoint: n1-1 down to n0
    int hist_n0;        // history slot 0 holds v^{hist_n0 - 1/2}; -1: no history
    int record;         // forward: write the seismograms
    int nt;             // steps of the whole run (adjoint memory bank parity)
};

__device__ __forceinline__ float* hist_slot(const ShotK& sh, int k)
{
    return sh.hist + (size_t)k * 2 * sh.g.nr * sh.g.P;
}

template <int N>
__device__ __forceinline__ const ShotK& shot_of(const ShotTable<N>& T, int4 tk)
{
    return T.s[N == 1 ? 0 : tk.x];
}

// pp: -1 the fields are updated in place (buffer 0); 0 / 1: read from
// buffer pp, written to the other (the launches of a fused step)
__device__ __forceinline__ ptrdiff_t field_in(const ShotK& sh, int pp)
{
    return pp == 1 ? (ptrdiff_t)sh.swap : 0;
}
__device__ __forceinline__ ptrdiff_t field_out(const ShotK& sh, int pp)
{
    return pp == 0 ? (ptrdiff_t)sh.swap : 0;
}

template <int N, int PM>
__device__ __forceinline__ void run_fwd_vel(const RunK& r, const ShotTable<N>& T, int n, int t,
                                            const BarK* bar, unsigned& epoch, FwdSmem& sm,
                                            int pp = -1)
{
    const int4 tk = r.tiles[t];
    const ShotK& sh = shot_of(T, tk);
    float* h0 = (r.hist_n0 >= 0 && n == r.hist_n0) ? hist_slot(sh, 0) : nullptr;
    fwd_vel_tile<PM>(sh.g, sh.C, sh.Sf, field_in(sh, pp), field_out(sh, pp), h0, tk.y, tk.z,
                     tk.w, bar, epoch, sm);
}

template <int N, int PM>
__device__ __forceinline__ void run_fwd_stress(const RunK& r, const ShotTable<N>& T, int n,
                                               int t, const BarK* bar, unsigned& epoch,
                                               FwdSmem& sm, int pp = -1)
{
    const int4 tk = r.tiles[t];
    const ShotK& sh = shot_of(T, tk);
    float* h = r.hist_n0 >= 0 ? hist_slot(sh, n - r.hist_n0 + 1) : nullptr;
    fwd_stress_tile<PM>(sh.g, sh.C, sh.Sf, field_in(sh, pp), field_out(sh, pp), sh.q, n,
                        r.record != 0, h, tk.y, tk.z, tk.w, bar, epoch, sm);
}

// forward tiles of either code variant (V 0: one path, 1: per tile class)
template <int N, int V>
__device__ __forceinline__ void run_fwd_vel_v(const RunK& r, const ShotTable<N>& T, int n, int t,
                                              const BarK* bar, unsigned& epoch, FwdSmem& sm)
{
    if (V == 0) run_fwd_vel<N, PM_ANY>(r, T, n, t, bar, epoch, sm);
    else if (r.tiles[t].w & TILE_PML) run_fwd_vel<N, PM_PML>(r, T, n, t, bar, epoch, sm);
    else run_fwd_vel<N, PM_INTERIOR>(r, T, n, t, bar, epoch, sm);
}

template <int N, int V>
__device__ __forceinline__ void run_fwd_stress_v(const RunK& r, const ShotTable<N>& T, int n,
                                                 int t, const BarK* bar, unsigned& epoch,
                                                 FwdSmem& sm)
{
    if (V == 0) run_fwd_stress<N, PM_ANY>(r, T, n, t, bar, epoch, sm);
    else if (r.tiles[t].w & TILE_PML) run_fwd_stress<N, PM_PML>(r, T, n, t, bar, epoch, sm);
    else run_fwd_stress<N, PM_INTERIOR>(r, T, n, t, bar, epoch, sm);
}

// statics / prefetch: the block keeps one tile for the whole run, so the
// velocity step of reverse step n stages the stress step's launch-invariant
// tiles for step n-1 (AdjSmem)
template <int N, bool RHO, int PM, typename SM>
__device__ __forceinline__ void run_adj_stress(const RunK& r, const ShotTable<N>& T, int n,
                                               int t, bool statics, bool defer,
                                               const BarK* bar, unsigned& epoch, SM& sm)
{
    const int4 tk = r.tiles[t];
    const ShotK& sh = shot_of(T, tk);
    const int parity = (r.nt - 1 - n) & 1;
    adj_stress_tile<RHO, PM>(sh.g, sh.C, sh.Sa[parity], sh.a, hist_slot(sh, n - r.hist_n0 + 1),
                    hist_slot(sh, n - r.hist_n0), tk.y, tk.z, tk.w, statics, defer, bar, epoch,
                    sm);
}

template <int N, bool RHO, int PM, bool PERSIST, typename SM>
__device__ __forceinline__ void run_adj_vel(const RunK& r, const ShotTable<N>& T, int n, int t,
                                            bool prefetch, bool deferred, const BarK* bar,
                                            unsigned& epoch, SM& sm)
{
    const int4 tk = r.tiles[t];
    const ShotK& sh = shot_of(T, tk);
    const int parity = (r.nt - 1 - n) & 1;
    // v^{n-1/2}: fcur of step n-1 (prefetch) and fprev of step n (deferred)
    const float* prev = hist_slot(sh, n - r.hist_n0);
    adj_vel_tile<RHO, PM, PERSIST>(sh.g, sh.C, sh.Sa[parity], sh.a, n, tk.y, tk.z, tk.w,
                      prefetch ? prev : nullptr,
                 deferred ? prev : nullptr, bar, epoch, sm);
}

// One launch per half-step: one block per tile, branching on the tile's
// class like the persistent kernels.  The per-class launches below (option
// "split") fit more interior blocks per SM; which is faster depends on the
// workload (the autotuner times both).
template <int N, int V>
__global__ void __launch_bounds__(kThreads, 5) k_fwd_vel(RunK r, int n,
                                                      const __grid_constant__ ShotTable<N> T)
{
    __shared__ FwdSmem sm;
    pdl_wait();
    unsigned epoch = 0;
    run_fwd_vel_v<N, V>(r, T, n, blockIdx.x, nullptr, epoch, sm);
    pdl_launch_dependents();
}

template <int N, int V>
__global__ void __launch_bounds__(kThreads, 5) k_fwd_stress(RunK r, int n,
                                                         const __grid_constant__ ShotTable<N> T)
{
    __shared__ FwdSmem sm;
    pdl_wait();
    unsigned epoch = 0;
    run_fwd_stress_v<N, V>(r, T, n, blockIdx.x, nullptr, epoch, sm);
    pdl_launch_dependents();
}

template <int N, bool RHO>
__global__ void __launch_bounds__(kThreads) k_adj_stress(RunK r, int n,
                                                         const __grid_constant__ ShotTable<N> T)
{
    __shared__ AdjSmem sm;
    pdl_wait();
    unsigned epoch = 0;
    if (r.tiles[blockIdx.x].w & TILE_PML)
        run_adj_stress<N, RHO, PM_PML>(r, T, n, blockIdx.x, false, false, nullptr, epoch, sm);
    else
        run_adj_stress<N, RHO, PM_INTERIOR>(r, T, n, blockIdx.x, false, false, nullptr, epoch, sm);
    pdl_launch_dependents();
}

template <int N, bool RHO>
__global__ void __launch_bounds__(kThreads) k_adj_vel(RunK r, int n,
                                                      const __grid_constant__ ShotTable<N> T)
{
    __shared__ AdjSmem sm;
    pdl_wait();
    unsigned epoch = 0;
    if (r.tiles[blockIdx.x].w & TILE_PML)
        run_adj_vel<N, RHO, PM_PML, false>(r, T, n, blockIdx.x, false, false, nullptr, epoch, sm);
    else
        run_adj_vel<N, RHO, PM_INTERIOR, false>(r, T, n, blockIdx.x, false, false, nullptr, epoch,
                                                sm);
    pdl_launch_dependents();
}

// One launch per half-step and tile class (option "split"): a launch of
// interior tiles carries no C-PML state and fits more blocks per SM (the
// velocity steps 8, the stress steps 6, C-PML tiles 5); it runs the same
// per-class tile code as the kernels above with the forward tile code 1.
template <int N, int PM>
__global__ void __launch_bounds__(kThreads, PM == PM_INTERIOR ? 8 : 5)
    k_fwd_vel_c(RunK r, int n, int pp, const __grid_constant__ ShotTable<N> T)
{
    __shared__ FwdSmem sm;
    pdl_wait();
    unsigned epoch = 0;
    run_fwd_vel<N, PM>(r, T, n, blockIdx.x, nullptr, epoch, sm, pp);
    pdl_launch_dependents();
}

template <int N, int PM>
__global__ void __launch_bounds__(kThreads, PM == PM_INTERIOR ? 6 : 5)
    k_fwd_stress_c(RunK r, int n, int pp, const __grid_constant__ ShotTable<N> T)
{
    __shared__ FwdSmem sm;
    pdl_wait();
    unsigned epoch = 0;
    run_fwd_stress<N, PM>(r, T, n, blockIdx.x, nullptr, epoch, sm, pp);
    pdl_launch_dependents();
}

template <int N, bool RHO, int PM>
__global__ void __launch_bounds__(kThreads, PM == PM_INTERIOR ? 6 : 5)
    k_adj_stress_c(RunK r, int n, const __grid_constant__ ShotTable<N> T)
{
    __shared__ typename std::conditional<PM == PM_INTERIOR, AdjStressIntSmem, AdjSmem>::type sm;
    pdl_wait();
    unsigned epoch = 0;
    run_adj_stress<N, RHO, PM>(r, T, n, blockIdx.x, false, false, nullptr, epoch, sm);
    pdl_launch_dependents();
}

template <int N, bool RHO, int PM>
__global__ void __launch_bounds__(kThreads, PM == PM_INTERIOR ? 8 : 5)
    k_adj_vel_c(RunK r, int n, const __grid_constant__ ShotTable<N> T)
{
    __shared__ AdjVelSmem<PM == PM_INTERIOR ? 4 : 8> sm;
    pdl_wait();
    unsigned epoch = 0;
    run_adj_vel<N, RHO, PM, false>(r, T, n, blockIdx.x, false, false, nullptr, epoch, sm);
    pdl_launch_dependents();
}

// ---------------------------------------------- pipelined interior tiles
//
// One launch per half-step over the interior tiles of a group, with a grid of
// a few blocks per SM: a block walks the tiles t, t + grid, t + 2 grid, ...
// and, while it computes one tile, the copies of its next tile are already
// in flight into the second of two shared-memory stages (cp.async groups,
// wait_group 1).  The own-node inputs travel the same way (each thread copies
// its own float4 groups), so nothing of the next tile waits on a register
// load.  The arithmetic is the shared core of the one-tile-per-block
// kernels, so the results agree with theirs bit for bit.

// one 16-byte copy of a thread's own group; zero-filled when !ok (src is
// then any valid address: nothing is read)
__device__ __forceinline__ void cp16(void* dst, const float* src, bool ok)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(ok ? 16u : 0u)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// all but the most recent group of this thread's copies have landed
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ V4 v4_of(const float4& f) { return V4{{f.x, f.y, f.z, f.w}}; }

struct __align__(16) VelStage {
    Tile a, b, c, d;           // trr, ttt, trz, tzz
    float4 own[4][kThreads];   // v_r, v_z, buoyancy at v_r and v_z of each thread's group
};

struct __align__(16) StressStage {
    Tile a, b;                 // v_r, v_z
    float4 own[7][kThreads];   // trr, ttt, tzz, trz, lambda, mu, harmonic mu
};

__device__ __forceinline__ void vel_issue(VelStage& b, const ShotK& sh, int i0, int j0)
{
    const WinK& g = sh.g;
    const StateK& S = sh.Sf;
    for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
        const Slot sl = slot_of(it, i0, j0, g);
        stage_async<EVEN>(b.a, S.trr, sl);
        stage_async<EVEN>(b.b, S.ttt, sl);
        stage_async<ODD>(b.c, S.trz, sl);
        stage_async<EVEN>(b.d, S.tzz, sl);
    }
    const Own o = own_of(g, i0, j0);
    const int tid = tid_of();
    const bool r1 = o.live && o.i >= 1;
    cp16(&b.own[0][tid], r1 ? S.vr + o.c : S.vr, r1);
    cp16(&b.own[1][tid], o.live ? S.vz + o.c : S.vz, o.live);
    cp16(&b.own[2][tid], r1 ? sh.C.w_bvr + o.cw : sh.C.w_bvr, r1);
    cp16(&b.own[3][tid], o.live ? sh.C.w_bvz + o.cw : sh.C.w_bvz, o.live);
}

__device__ __forceinline__ void stress_issue(StressStage& b, const ShotK& sh, int i0, int j0)
{
    const WinK& g = sh.g;
    const StateK& S = sh.Sf;
    const CoefK& C = sh.C;
    for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
        const Slot sl = slot_of(it, i0, j0, g);
        stage_async<ODD>(b.a, S.vr, sl);
        stage_async<EVEN>(b.b, S.vz, sl);
    }
    const Own o = own_of(g, i0, j0);
    const int tid = tid_of();
    const bool r1 = o.live && o.i >= 1;
    cp16(&b.own[0][tid], o.live ? S.trr + o.c : S.trr, o.live);
    cp16(&b.own[1][tid], o.live ? S.ttt + o.c : S.ttt, o.live);
    cp16(&b.own[2][tid], o.live ? S.tzz + o.c : S.tzz, o.live);
    cp16(&b.own[3][tid], r1 ? S.trz + o.c : S.trz, r1);
    cp16(&b.own[4][tid], o.live ? C.w_lam + o.cw : C.w_lam, o.live);
    cp16(&b.own[5][tid], o.live ? C.w_mu + o.cw : C.w_mu, o.live);
    cp16(&b.own[6][tid], r1 ? C.w_muh + o.cw : C.w_muh, r1);
}

// negate this thread's staged slots of an odd field that are mirror rows
__device__ __forceinline__ void negate_mirror(Tile& t, int i0, int j0, const WinK& g)
{
    if (i0 < kH) {
        for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
            const Slot sl = slot_of(it, i0, j0, g);
            if (sl.neg && sl.off_o >= 0) negate_slot(t, sl);
        }
    }
}

template <int N>
__global__ void __launch_bounds__(kThreads, 4)
    k_fwd_vel_pipe(RunK r, int n, const __grid_constant__ ShotTable<N> T)
{
    __shared__ VelStage st[2];
    pdl_wait();
    unsigned epoch = 0;
    int t = blockIdx.x;
    if (t < r.ntiles) {
        const int4 tk = r.tiles[t];
        vel_issue(st[0], shot_of(T, tk), tk.y, tk.z);
    }
    cp_commit();
    for (int k = 0; t < r.ntiles; ++k, t += gridDim.x) {
        const int tn = t + (int)gridDim.x;
        if (tn < r.ntiles) {
            const int4 tk = r.tiles[tn];
            vel_issue(st[(k + 1) & 1], shot_of(T, tk), tk.y, tk.z);
        }
        cp_commit();
        cp_wait_prev();
        VelStage& b = st[k & 1];
        const int4 tk = r.tiles[t];
        const ShotK& sh = shot_of(T, tk);
        const WinK& g = sh.g;
        negate_mirror(b.c, tk.y, tk.z, g);
        __syncthreads();
        const Own o = own_of(g, tk.y, tk.z);
        const int tid = tid_of();
        const V4 vr0 = v4_of(b.own[0][tid]), vz0 = v4_of(b.own[1][tid]);
        const V4 br = v4_of(b.own[2][tid]);
        V4 bz = v4_of(b.own[3][tid]);
        float ivr = 0.f, ivh = 0.f;
        if (o.live) {
            ivr = __ldg(sh.C.inv_r_int + o.i);
            ivh = __ldg(sh.C.inv_r_half + o.i);
            if (tk.w & TILE_LAST) patch4(bz, o.j, g.nz - 1, bvz_at(sh.C, g, o.i, g.nz - 1));
        }
        float* h0 = (r.hist_n0 >= 0 && n == r.hist_n0) ? hist_slot(sh, 0) : nullptr;
        const V4 zero{};
        fwd_vel_core<PM_INTERIOR>(g, sh.Sf, 0, h0, o, false, vr0, vz0, br, bz, zero, zero, zero,
                                  zero, ivr, ivh, b.a, b.b, b.c, b.d, nullptr, nullptr, epoch);
        __syncthreads();  // stage k & 1 is refilled at the next iteration
    }
    pdl_launch_dependents();
}

template <int N>
__global__ void __launch_bounds__(kThreads, 4)
    k_fwd_stress_pipe(RunK r, int n, const __grid_constant__ ShotTable<N> T)
{
    __shared__ StressStage st[2];
    pdl_wait();
    unsigned epoch = 0;
    int t = blockIdx.x;
    if (t < r.ntiles) {
        const int4 tk = r.tiles[t];
        stress_issue(st[0], shot_of(T, tk), tk.y, tk.z);
    }
    cp_commit();
    for (int k = 0; t < r.ntiles; ++k, t += gridDim.x) {
        const int tn = t + (int)gridDim.x;
        if (tn < r.ntiles) {
            const int4 tk = r.tiles[tn];
            stress_issue(st[(k + 1) & 1], shot_of(T, tk), tk.y, tk.z);
        }
        cp_commit();
        cp_wait_prev();
        StressStage& b = st[k & 1];
        const int4 tk = r.tiles[t];
        const ShotK& sh = shot_of(T, tk);
        const WinK& g = sh.g;
        negate_mirror(b.a, tk.y, tk.z, g);
        __syncthreads();
        const Own o = own_of(g, tk.y, tk.z);
        const int tid = tid_of();
        const V4 t_rr = v4_of(b.own[0][tid]), t_tt = v4_of(b.own[1][tid]);
        const V4 t_zz = v4_of(b.own[2][tid]), t_rz = v4_of(b.own[3][tid]);
        const V4 lm = v4_of(b.own[4][tid]), mu = v4_of(b.own[5][tid]);
        V4 mh = v4_of(b.own[6][tid]);
        float ivh = 0.f;
        if (o.live) {
            ivh = __ldg(sh.C.inv_r_half + o.i);
            if (o.i >= 1 && (tk.w & TILE_LAST))
                patch4(mh, o.j, g.nz - 1, muh_at(sh.C, g, o.i, g.nz - 1));
        }
        float* h = r.hist_n0 >= 0 ? hist_slot(sh, n - r.hist_n0 + 1) : nullptr;
        const V4 zero{};
        fwd_stress_core<PM_INTERIOR>(g, sh.Sf, 0, sh.q, n, r.record != 0, h, o, false, t_rr, t_tt,
                                     t_zz, t_rz, lm, mu, mh, zero, zero, zero, zero, ivh, b.a,
                                     b.b, nullptr, nullptr, epoch);
        __syncthreads();
    }
    pdl_launch_dependents();
}

// ------------------------------------------------- fused interior steps
//
// One launch per time step over the interior tiles (option "split" 3): both
// half-steps of Eq. 2 for a tile.  The block updates v at the nodes its
// stress stencils read (v_r rows i0-1 .. i0+17, v_z rows i0-2 .. i0+16,
// columns j0-4 .. j0+35 in float4 groups) and keeps them in shared memory,
// then runs the stress half-step of its own nodes, so the wavefields cross
// HBM once per step instead of once per half-step.  Those velocity updates
// read tau^n on rows i0-3 .. i0+18 and columns j0-8 .. j0+39 (staged),
// v^{n-1/2} and the buoyancies on the usual 2-node halo.
// Neighbouring tiles recompute each other's halo velocities, which is why
// the fields ping-pong: the launch reads buffer pp and writes buffer 1 - pp,
// and the C-PML tiles of the same step run the two half-step launches on
// the same buffers.  An interior tile's 2-node-halo region holds no C-PML
// node and lies inside the window (the layers are between it and every
// edge but the axis), so its halo velocities need no layer state and no
// zero edge; the axis mirror is applied to the updated velocities.  The
// arithmetic is that of the half-step kernels, node for node.

constexpr int kTop4 = 3;                // staged rows i0-3 .. i0+18
constexpr int kSR4 = kTR + kTop4 + 3;  // 22
constexpr int kSZ4 = kTZ + 16;       // 48 staged columns, j0-8 .. j0+39
constexpr int kQ4 = kSZ4 / 4;
typedef float Tile4[kSR4][kSZ4];

__device__ __forceinline__ V4 lds4(const Tile4& s, int rr, int cc)
{
    const float4 t = *reinterpret_cast<const float4*>(&s[rr][cc]);
    return V4{{t.x, t.y, t.z, t.w}};
}

__device__ __forceinline__ V12 lds12(const Tile4& s, int rr, int cc)
{
    V12 r;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 t = *reinterpret_cast<const float4*>(&s[rr][cc + 4 * k]);
        r.v[4 * k] = t.x;
        r.v[4 * k + 1] = t.y;
        r.v[4 * k + 2] = t.z;
        r.v[4 * k + 3] = t.w;
    }
    return r;
}

// the slot geometry of slot_of for the 4-node-halo staging
__device__ __forceinline__ Slot slot4_of(int it, int i0, int j0, const WinK& g)
{
    Slot s;
    s.rr = it / kQ4;
    s.cq = 4 * (it - s.rr * kQ4);
    const int i = i0 - kTop4 + s.rr, j = j0 - 8 + s.cq;
    const bool zin = j >= 0 && j < g.nz;
    s.zlim = zin ? min(4, g.nz - j) : 0;
    const int ie = i < 0 ? -1 - i : i;
    const int io = i < 0 ? -i : i;
    s.neg = i < 0;
    s.off_e = (zin && ie < g.nr) ? ie * g.P + j : -1;
    s.off_o = (zin && io >= 1 && io < g.nr) ? io * g.P + j : -1;
    s.offw_e = s.offw_o = -1;
    return s;
}

template <int KIND>
__device__ __forceinline__ void stage4_async(Tile4& t, const float* __restrict__ f, const Slot& s)
{
    const int off = KIND == EVEN ? s.off_e : s.off_o;
    const float* src = f + (off >= 0 ? off : 0);
    const unsigned bytes = off >= 0 ? 4u * (unsigned)s.zlim : 0u;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(&t[s.rr][s.cq])),
                 "l"(src), "r"(bytes)
                 : "memory");
}

struct __align__(128) StepSmem {
    Tile4 rr, tt, zz, rz;  // tau^n
    Tile vr, vz;           // v^{n-1/2}, replaced by v^{n+1/2}
    Tile br, bz;           // buoyancy at the v_r and v_z nodes
};

// The part of a fused interior step after the staging: the velocity
// updates on the halo region, the axis mirror of the result, the own
// velocities and history, and the stress half-step of the own nodes.
template <int N>
__device__ __forceinline__ void fused_step_tail(const RunK& r, int n, const ShotK& sh,
                                                ptrdiff_t fout, const Own& o, const V4& lm,
                                                const V4& mu, const V4& mh, float ivh,
                                                StepSmem& sm)
{
    const WinK& g = sh.g;
    const CoefK& C = sh.C;
    const StateK& S = sh.Sf;
    const int4 tk = r.tiles[blockIdx.x];
    const int i0 = tk.y;
    // v^{n-1/2} of the own nodes (history slot 0 of a segment's first step)
    const bool h0 = r.hist_n0 >= 0 && n == r.hist_n0;
    V4 vr_old{}, vz_old{};
    if (h0) {
        vr_old = lds4(sm.vr, o.rr, o.cc);
        vz_old = lds4(sm.vz, o.rr, o.cc);
    }
    __syncthreads();
    // ---- velocity half-step at the nodes the stress stencils read (rows
    // i >= 0; the mirror rows follow), in place over this thread's slots:
    // v_r on staged rows 1 .. 19, v_z on rows 0 .. 18
    for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
        const int r2 = it / kQ, c2 = 4 * (it - r2 * kQ);
        const int i = i0 - kH + r2;
        if (i < 0) continue;
        const int R = r2 + (kTop4 - kH), K = c2 + 4;  // the same node in the Tile4 grid
        const V12 rz12 = lds12(sm.rz, R, K - 4);
        if (i >= 1 && r2 >= 1) {
            const V4 rm2 = lds4(sm.rr, R - 2, K), rm1 = lds4(sm.rr, R - 1, K);
            const V4 r0 = lds4(sm.rr, R, K), rp1 = lds4(sm.rr, R + 1, K);
            const V4 tm1 = lds4(sm.tt, R - 1, K), t0 = lds4(sm.tt, R, K);
            const V4 vr0 = lds4(sm.vr, r2, c2), br = lds4(sm.br, r2, c2);
            const float inv_r = __ldg(C.inv_r_int + i);
            float vr[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float d_trr = d4(r0.v[e], rm1.v[e], rp1.v[e], rm2.v[e]) * g.inv_dr;
                float d_trz = d4(rz12.v[4 + e], rz12.v[3 + e], rz12.v[5 + e], rz12.v[2 + e]) * g.inv_dz;
                const float hoop = 0.5f * ((rm1.v[e] - tm1.v[e]) + (r0.v[e] - t0.v[e])) * inv_r;
                vr[e] = vr0.v[e] + g.dt * br.v[e] * (d_trr + d_trz + hoop);
            }
            *reinterpret_cast<float4*>(&sm.vr[r2][c2]) = make_float4(vr[0], vr[1], vr[2], vr[3]);
        }
        if (r2 < kSR - 1) {
            const V12 zz12 = lds12(sm.zz, R, K - 4);
            const V4 rzp1 = lds4(sm.rz, R + 1, K);
            const V4 rzm1 = lds4(sm.rz, R - 1, K), rzp2 = lds4(sm.rz, R + 2, K);
            const V4 vz0 = lds4(sm.vz, r2, c2), bz = lds4(sm.bz, r2, c2);
            const float inv_r = __ldg(C.inv_r_half + i);
            float vz[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float d_trz = d4(rzp1.v[e], rz12.v[4 + e], rzp2.v[e], rzm1.v[e]) * g.inv_dr;
                float d_tzz = d4(zz12.v[5 + e], zz12.v[4 + e], zz12.v[6 + e], zz12.v[3 + e]) * g.inv_dz;
                const float hoop = 0.5f * (rz12.v[4 + e] + rzp1.v[e]) * inv_r;
                vz[e] = vz0.v[e] + g.dt * bz.v[e] * (d_trz + d_tzz + hoop);
            }
            *reinterpret_cast<float4*>(&sm.vz[r2][c2]) = make_float4(vz[0], vz[1], vz[2], vz[3]);
        }
    }
    __syncthreads();
    if (i0 < kH) {
        // mirror rows of the axis tile: v_r odd (v_r[-k] = -v_r[k]), v_z even
        // (v_z[-1-k] = v_z[k])
        const int it = tid_of();
        if (it < kH * kQ) {
            const int r2 = it / kQ, c2 = 4 * (it - r2 * kQ);
            const int i = i0 - kH + r2;  // -2 or -1
            const float4 a = *reinterpret_cast<const float4*>(&sm.vr[r2 - 2 * i][c2]);
            const float4 b = *reinterpret_cast<const float4*>(&sm.vz[r2 - 2 * i - 1][c2]);
            *reinterpret_cast<float4*>(&sm.vr[r2][c2]) = make_float4(-a.x, -a.y, -a.z, -a.w);
            *reinterpret_cast<float4*>(&sm.vz[r2][c2]) = b;
        }
        __syncthreads();
    }
    if (o.live) {
        const V4 a = lds4(sm.vr, o.rr, o.cc), b = lds4(sm.vz, o.rr, o.cc);
        if (o.i >= 1) st4(S.vr + fout + o.c, o.j, g.nz, a.v);
        st4(S.vz + fout + o.c, o.j, g.nz, b.v);
        if (h0) {
            float* hs = hist_slot(sh, 0);
            st4(hs + o.c, o.j, g.nz, vr_old.v);
            st4(hs + g.nr * g.P + o.c, o.j, g.nz, vz_old.v);
        }
    }
    // ---- stress half-step of the own nodes
    const int R = o.rr + (kTop4 - kH), K = o.cc + 4;
    const V4 t_rr = lds4(sm.rr, R, K), t_tt = lds4(sm.tt, R, K), t_zz = lds4(sm.zz, R, K);
    const V4 t_rz = lds4(sm.rz, R, K);
    float* h = r.hist_n0 >= 0 ? hist_slot(sh, n - r.hist_n0 + 1) : nullptr;
    const V4 zero{};
    unsigned epoch = 0;
    fwd_stress_core<PM_INTERIOR>(g, S, fout, sh.q, n, r.record != 0, h, o, false, t_rr, t_tt,
                                 t_zz, t_rz, lm, mu, mh, zero, zero, zero, zero, ivh, sm.vr,
                                 sm.vz, nullptr, nullptr, epoch);
}

template <int N>
__global__ void __launch_bounds__(kThreads, 6)
    k_fwd_step(RunK r, int n, int pp, const __grid_constant__ ShotTable<N> T)
{
    __shared__ StepSmem sm;
    pdl_wait();
    const int4 tk = r.tiles[blockIdx.x];
    const ShotK& sh = shot_of(T, tk);
    const WinK& g = sh.g;
    const CoefK& C = sh.C;
    const StateK& S = sh.Sf;
    const ptrdiff_t fin = field_in(sh, pp), fout = field_out(sh, pp);
    const int i0 = tk.y, j0 = tk.z;
    const Own o = own_of(g, i0, j0);
    for (int it = tid_of(); it < kSR4 * kQ4; it += kThreads) {
        const Slot sl = slot4_of(it, i0, j0, g);
        stage4_async<EVEN>(sm.rr, S.trr + fin, sl);
        stage4_async<EVEN>(sm.tt, S.ttt + fin, sl);
        stage4_async<EVEN>(sm.zz, S.tzz + fin, sl);
        stage4_async<ODD>(sm.rz, S.trz + fin, sl);
    }
    for (int it = tid_of(); it < kSR * kQ; it += kThreads) {
        const Slot sl = slot_of(it, i0, j0, g);
        stage_async<ODD>(sm.vr, S.vr + fin, sl);
        stage_async<EVEN>(sm.vz, S.vz + fin, sl);
        stage_async<ABS, true>(sm.br, C.w_bvr, sl);
        stage_async<EVEN, true>(sm.bz, C.w_bvz, sl);
    }
    // own-node inputs of the stress half-step, in flight with the copies
    V4 lm{}, mu{}, mh{};
    float ivh = 0.f;
    if (o.live) {
        ivh = __ldg(C.inv_r_half + o.i);
        lm = ld4g(C.w_lam + o.cw);
        mu = ld4g(C.w_mu + o.cw);
        if (o.i >= 1) mh = ld4g(C.w_muh + o.cw);
    }
    async_wait_all();
    if (i0 < kTop4) {
        for (int it = tid_of(); it < kSR4 * kQ4; it += kThreads) {
            const Slot sl = slot4_of(it, i0, j0, g);
            if (sl.neg && sl.off_o >= 0) {
                float4* q = reinterpret_cast<float4*>(&sm.rz[sl.rr][sl.cq]);
                float4 v = *q;
                v.x = -v.x;
                v.y = -v.y;
                v.z = -v.z;
                v.w = -v.w;
                *q = v;
            }
        }
    }
    __syncthreads();
    fused_step_tail<N>(r, n, sh, fout, o, lm, mu, mh, ivh, sm);
    pdl_launch_dependents();
}

// ------------------------------------ fused interior steps, TMA staging
//
// The same fused step (option "split" 4) with its eight tiles staged by the
// tensor memory accelerator: one thread issues a 2-D box copy per field
// (cp.async.bulk.tensor, 3-D tensor maps over the shots' field planes and
// over the coefficient copies, no multicast) that completes on a shared
// mbarrier, instead of 128 threads issuing 16-byte cp.async copies slot by
// slot.  Interior tiles lie inside their window, so the boxes need no zero
// edge; rows above the axis come back zero-filled and the axis tile
// rebuilds the stresses' mirror rows from the copied ones (the velocity
// and buoyancy mirror rows are never read).  Every box starts at a column
// that is a multiple of 4 floats (tile columns are multiples of 32, the
// coefficient copies are shifted for that), every destination tile is
// 128-byte aligned.  The wait is bounded: a copy that does not complete
// sets *err, and the block returns.

struct TmaMaps {
    CUtensorMap t[2];  // stresses of field buffer 0 / 1 (planes shot * 14 + f / shot * 6 + f), box 48 x 22
    CUtensorMap v[2];  // velocities of field buffer 0 / 1, box 40 x 20
    CUtensorMap w;     // coefficient copies (planes 5 k + q), box 40 x 20
};

constexpr unsigned kStepTmaBytes = 4u * kSR4 * kSZ4 * 4u + 4u * kSR * kSZ * 4u;

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for phase `parity` of the mbarrier
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity)
{
    for (int k = 0; k < (1 << 22); ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

template <int N>
__global__ void __launch_bounds__(kThreads, 6)
    k_fwd_step_tma(RunK r, int n, int pp, int s0, int* err, const __grid_constant__ TmaMaps M,
                   const __grid_constant__ ShotTable<N> T)
{
    __shared__ StepSmem sm;
    __shared__ __align__(8) unsigned long long mbar;
    const unsigned bar = smem_addr(&mbar);
    const int tid = tid_of();
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    pdl_wait();
    const int4 tk = r.tiles[blockIdx.x];
    const ShotK& sh = shot_of(T, tk);
    const WinK& g = sh.g;
    const CoefK& C = sh.C;
    const ptrdiff_t fout = field_out(sh, pp);
    const int i0 = tk.y, j0 = tk.z;
    const Own o = own_of(g, i0, j0);
    if (tid == 0) {
        mbar_expect_tx(bar, kStepTmaBytes);
        const int b = pp == 1 ? 1 : 0;  // the buffer this step reads
        const int shot = s0 + tk.x;
        const int base = b ? shot * 6 : shot * 14;  // plane of v_r; v_z, trr, ttt, tzz, trz follow
        const CUtensorMap* mt = &M.t[b];
        const CUtensorMap* mv = &M.v[b];
        tma_load_3d(&sm.rr, mt, j0 - 8, i0 - kTop4, base + 2, bar);
        tma_load_3d(&sm.tt, mt, j0 - 8, i0 - kTop4, base + 3, bar);
        tma_load_3d(&sm.zz, mt, j0 - 8, i0 - kTop4, base + 4, bar);
        tma_load_3d(&sm.rz, mt, j0 - 8, i0 - kTop4, base + 5, bar);
        tma_load_3d(&sm.vr, mv, j0 - 4, i0 - kH, base + 0, bar);
        tma_load_3d(&sm.vz, mv, j0 - 4, i0 - kH, base + 1, bar);
        const int kc = (4 - (g.z0 & 3)) & 3;  // the shifted copy of this window
        tma_load_3d(&sm.br, &M.w, g.z0 + kc + j0 - 4, i0 - kH, 5 * kc + 3, bar);
        tma_load_3d(&sm.bz, &M.w, g.z0 + kc + j0 - 4, i0 - kH, 5 * kc + 4, bar);
    }
    // own-node inputs of the stress half-step, in flight with the copies
    V4 lm{}, mu{}, mh{};
    float ivh = 0.f;
    if (o.live) {
        ivh = __ldg(C.inv_r_half + o.i);
        lm = ld4g(C.w_lam + o.cw);
        mu = ld4g(C.w_mu + o.cw);
        if (o.i >= 1) mh = ld4g(C.w_muh + o.cw);
    }
    if (!mbar_wait_bounded(bar, 0)) {
        if (tid == 0) atomicExch(err, 1);
        mbar_wait_bounded(bar, 0);  // the copies still in flight, once more, bounded
        return;
    }
    if (i0 < kTop4) {
        // the axis tile: stresses at rows i < 0 from their mirror images
        // (cells even, f[-1-k] = f[k]; trz odd, f[-k] = -f[k])
        for (int it = tid; it < 4 * kTop4 * kQ4; it += kThreads) {
            const int f = it / (kTop4 * kQ4), q = it - f * (kTop4 * kQ4);
            const int rr = q / kQ4, cq = 4 * (q - rr * kQ4);
            Tile4& t = f == 0 ? sm.rr : f == 1 ? sm.tt : f == 2 ? sm.zz : sm.rz;
            const int i = rr - kTop4;  // -3 .. -1
            const float4 src = *reinterpret_cast<const float4*>(
                &t[(f == 3 ? -i : -1 - i) + kTop4][cq]);
            *reinterpret_cast<float4*>(&t[rr][cq]) =
                f == 3 ? make_float4(-src.x, -src.y, -src.z, -src.w) : src;
        }
    }
    __syncthreads();
    fused_step_tail<N>(r, n, sh, fout, o, lm, mu, mh, ivh, sm);
    pdl_launch_dependents();
}

// every step n0 .. n1-1 of every shot of the table in one cooperative launch
template <int N, int V>
__global__ void __launch_bounds__(kThreads, 5) k_fwd_persist(RunK r, BarK b,
                                                             const __grid_constant__ ShotTable<N> T)
{
    __shared__ FwdSmem sm;
    unsigned epoch = 0;
    const bool idle = (int)blockIdx.x >= r.ntiles;
    for (int n = r.n0; n < r.n1; ++n) {
        // the block's last tile of a phase arrives at the barrier itself
        for (int t = blockIdx.x; t < r.ntiles; t += gridDim.x)
            run_fwd_vel_v<N, V>(r, T, n, t, t + (int)gridDim.x >= r.ntiles ? &b : nullptr, epoch,
                                sm);
        if (idle) grid_arrive(b, epoch);
        if (!grid_wait(b, epoch)) return;
        for (int t = blockIdx.x; t < r.ntiles; t += gridDim.x)
            run_fwd_stress_v<N, V>(r, T, n, t, t + (int)gridDim.x >= r.ntiles ? &b : nullptr,
                                   epoch, sm);
        if (idle) grid_arrive(b, epoch);
        if (!grid_wait(b, epoch)) return;
    }
}

// reverse steps n1-1 down to n0 of every shot of the table in one cooperative launch
template <int N, bool RHO>
__global__ void __launch_bounds__(kThreads, 5) k_adj_persist(RunK r, BarK b,
                                                             const __grid_constant__ ShotTable<N> T)
{
    __shared__ AdjSmem sm;
    unsigned epoch = 0;
    const bool one = r.ntiles <= (int)gridDim.x;  // at most one tile per block
    const bool idle = (int)blockIdx.x >= r.ntiles;
    for (int n = r.n1 - 1; n >= r.n0; --n) {
        // the block's last tile of a phase arrives at the barrier itself
        for (int t = blockIdx.x; t < r.ntiles; t += gridDim.x) {
            const BarK* bb = t + (int)gridDim.x >= r.ntiles ? &b : nullptr;
            const bool st = one && n < r.n1 - 1;
            if (r.tiles[t].w & TILE_PML)
                run_adj_stress<N, RHO, PM_PML>(r, T, n, t, st, one, bb, epoch, sm);
            else
                run_adj_stress<N, RHO, PM_INTERIOR>(r, T, n, t, st, one, bb, epoch, sm);
        }
        if (idle) grid_arrive(b, epoch);
        if (!grid_wait(b, epoch)) return;
        for (int t = blockIdx.x; t < r.ntiles; t += gridDim.x) {
            const BarK* bb = t + (int)gridDim.x >= r.ntiles ? &b : nullptr;
            const bool pf = one && n > r.n0;
            if (r.tiles[t].w & TILE_PML)
                run_adj_vel<N, RHO, PM_PML, true>(r, T, n, t, pf, one, bb, epoch, sm);
            else
                run_adj_vel<N, RHO, PM_INTERIOR, true>(r, T, n, t, pf, one, bb, epoch, sm);
        }
        if (idle) grid_arrive(b, epoch);
        if (!grid_wait(b, epoch)) return;
    }
}

// transpose of the recording at the last step of one shot: dp[nt-1]/3 into
// each normal stress of the receiver cells
__global__ void k_adj_inject(const __grid_constant__ ShotK sh, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= sh.g.nz) return;
    const int r = sh.a.recmap[k];
    if (r < 0) return;
    const StateK& S = sh.Sa[0];
    const float r3 = sh.a.resid[(size_t)r * sh.a.nt + n] * (1.f / 3.f);
    S.trr[k] += r3;
    S.ttt[k] += r3;
    S.tzz[k] += r3;
}

// ------------------------------------------------------------ finalise

struct FinK {
    double *g_lam, *g_mu, *g_rho, *H_lam, *H_mu;  // global [nr][nzg], accumulated
};

__device__ __forceinline__ double kval(const float2* a, size_t k)
{
    float2 s = a[k];
    return (double)s.x - (double)s.y;
}

// Chain rule from the node accumulators of one shot to per-cell gradients,
// added into the global FP64 arrays.  Cells of the window's C-PML get nothing.
__global__ void k_finalize(const __grid_constant__ ShotK sh, FinK f)
{
    const WinK& g = sh.g;
    const CoefK& C = sh.C;
    const AdjK& q = sh.a;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nr - g.npml_r || j < g.npml_z || j >= g.nz - g.npml_z) return;
    const size_t c = (size_t)i * g.P + j;
    const size_t cg = (size_t)i * g.nzg + g.z0 + j;
    const double mu = C.mu[cg], rho = C.rho[cg];

    double gl = kval(q.G_lam, c);
    double gm = kval(q.G_munn, c);
    double hl = q.H_lam[c];
    double hm = q.H_munn[c];
    // the four shear nodes around the cell: rows i, i+1; columns j-1, j
    for (int di = 0; di < 2; ++di) {
        int ii = i + di;
        if (ii < 1 || ii >= g.nr) continue;
        for (int dj = -1; dj <= 0; ++dj) {
            int jj = j + dj;
            if (jj < 0) continue;
            // the window's last node row averages its own cells twice
            const double mult = (jj == g.nz - 1) ? 2.0 : 1.0;
            size_t k = (size_t)ii * g.P + jj;
            double mh = muh_at(C, g, ii, jj);
            if (mh > 0.0) gm += mult * mh * mh / (4.0 * mu * mu) * kval(q.G_murz, k);
            hm += mult * 0.25 * (double)q.H_murz[k];
        }
    }
    // plain adds (no fused multiply-add into the running sums): the sum over
    // shots rounds the same way however the shots are batched
    f.g_lam[cg] = __dadd_rn(f.g_lam[cg], gl);
    f.g_mu[cg] = __dadd_rn(f.g_mu[cg], gm);
    f.H_lam[cg] = __dadd_rn(f.H_lam[cg], hl);
    f.H_mu[cg] = __dadd_rn(f.H_mu[cg], hm);
    if (f.g_rho) {
        // buoyancy nodes that average this cell: v_r rows i, i+1; v_z columns j-1, j
        double gb = 0.0;
        for (int di = 0; di < 2; ++di) {
            int ii = i + di;
            if (ii < 1 || ii >= g.nr) continue;
            size_t k = (size_t)ii * g.P + j;
            gb += kval(q.G_br, k) / (double)C.bvr[(size_t)ii * g.nzg + g.z0 + j];
        }
        for (int dj = -1; dj <= 0; ++dj) {
            int jj = j + dj;
            if (jj < 0) continue;
            const double mult = (jj == g.nz - 1) ? 2.0 : 1.0;
            size_t k = (size_t)i * g.P + jj;
            gb += mult * kval(q.G_bz, k) / (double)bvz_at(C, g, i, jj);
        }
        f.g_rho[cg] = __dadd_rn(f.g_rho[cg], __dmul_rn(-0.5 / (rho * rho), gb));
    }
}

}  // namespace bh
