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
#include <cuda_runtime.h>
#include <stdint.h>

namespace bh {

constexpr float kC1 = 1.125f;              // 9/8
constexpr float kC2 = -0.041666666666666664f; // -1/24

struct WinK {
    int nr, nz, P;      // window rows, columns, row pitch of the state arrays
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
// 32 columns of z).  A block of 256 threads (8 warps) first stages what the
// tile's stencils read, tile plus a 2-node halo, into shared memory (warp w
// stages rows w, w+8, w+16, one row per pass so that row-level decisions --
// axis mirror, outer edge -- are warp-uniform), with the mirror and the zero
// edges applied; then warp w computes rows w and w+8 of the tile, one column
// per lane.  The adjoint tiles also build the transposed-stencil
// coefficients once per staged node.
//
// The same tile functions serve two launch forms: one kernel per half-step
// (one tile per block), and one persistent cooperative kernel per shot that
// runs every time step, with a bounded grid barrier between half-steps.
// State written inside a launch is read with ld.global.cg (L2, not the
// SM-private L1, which other SMs' writes do not update).
constexpr int kTZ = 32, kTR = 16, kH = 2;
constexpr int kSZ = kTZ + 2 * kH, kSR = kTR + 2 * kH;
constexpr int kThreads = 256;
typedef float Tile[kSR][kSZ];

// Programmatic dependent launch: a kernel may be scheduled while its
// predecessor drains; it must wait here before touching the predecessor's
// outputs.  No-op when launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

// Stage the tile's rows [i0-2, i0+18) x columns [j0-2, j0+34) of a window
// field.  EVEN: half-r field (cells, v_z), mirror f[-1-k] = f[k].  ODD:
// integer-r field (v_r, trz), f[-k] = -f[k], f[0] = 0.  Zero beyond nr and
// outside 0 <= z < nz.
enum { EVEN = 0, ODD = 1 };
template <int KIND>
__device__ __forceinline__ void stage(Tile& s, const float* __restrict__ f, int i0, int j0,
                                      const WinK& g)
{
    const int lane = threadIdx.x;
    for (int rr = threadIdx.y; rr < kSR; rr += 8) {
        int i = i0 - kH + rr;
        float sg = 1.f;
        if (KIND == EVEN) {
            if (i < 0) i = -1 - i;
        } else {
            if (i < 0) { i = -i; sg = -1.f; }
            if (i == 0) sg = 0.f;
        }
        const bool live = i < g.nr && sg != 0.f;
        const float* row = f + (live ? i * g.P : 0);
        int j = j0 - kH + lane;
        s[rr][lane] = (live && j >= 0 && j < g.nz) ? sg * ldcg(row + j) : 0.f;
        if (lane < kSZ - 32) {
            j += 32;
            s[rr][lane + 32] = (live && j < g.nz) ? sg * ldcg(row + j) : 0.f;
        }
    }
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

struct FwdSmem {
    Tile a, b, c, d;
};

// Velocity half-step of one tile: Eq. 2 lines 1-2 with the C-PML memories 0..3.
// Every own-node input is loaded into registers before the staging, so the
// tile pays one round trip to L2 (the loads and stores go through pointers
// the compiler must assume may alias, so it would not reorder them itself).
__device__ __forceinline__ void fwd_vel_tile(const WinK& g, const CoefK& C, const StateK& S,
                                             float* hist0, int i0, int j0, FwdSmem& sm)
{
    Tile &s_rr = sm.a, &s_tt = sm.b, &s_rz = sm.c, &s_zz = sm.d;
    const int j = j0 + threadIdx.x, zz = threadIdx.x + kH;
    const bool jok = j < g.nz;
    float vr0[2], vz0[2], br[2], bz[2], q0[2], q1[2], q2[2], q3[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int i = i0 + threadIdx.y + 8 * p;
        vr0[p] = vz0[p] = br[p] = bz[p] = q0[p] = q1[p] = q2[p] = q3[p] = 0.f;
        if (jok && i < g.nr) {
            const int c = i * g.P + j;
            vz0[p] = ldcg(S.vz + c);
            bz[p] = bvz_at(C, g, i, j);
            if (C.ar_half[i] != 0.f) q2[p] = ldcg(S.psi[2] + c);
            if (C.az_half[j] != 0.f) q3[p] = ldcg(S.psi[3] + c);
            if (i >= 1) {
                vr0[p] = ldcg(S.vr + c);
                br[p] = __ldg(C.bvr + (size_t)i * g.nzg + g.z0 + j);
                if (C.ar_int[i] != 0.f) q0[p] = ldcg(S.psi[0] + c);
                if (C.az_int[j] != 0.f) q1[p] = ldcg(S.psi[1] + c);
            }
        }
    }
    __syncthreads();
    stage<EVEN>(s_rr, S.trr, i0, j0, g);
    stage<EVEN>(s_tt, S.ttt, i0, j0, g);
    stage<ODD>(s_rz, S.trz, i0, j0, g);
    stage<EVEN>(s_zz, S.tzz, i0, j0, g);
    __syncthreads();
    if (!jok) return;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int i = i0 + threadIdx.y + 8 * p, rr = threadIdx.y + 8 * p + kH;
        if (i >= g.nr) break;
        const int c = i * g.P + j;
        if (i >= 1) {
            float d_trr = d4(s_rr[rr][zz], s_rr[rr - 1][zz], s_rr[rr + 1][zz], s_rr[rr - 2][zz]) *
                          g.inv_dr;
            float d_trz = d4(s_rz[rr][zz], s_rz[rr][zz - 1], s_rz[rr][zz + 1], s_rz[rr][zz - 2]) *
                          g.inv_dz;
            float hoop = 0.5f * ((s_rr[rr - 1][zz] - s_tt[rr - 1][zz]) + (s_rr[rr][zz] - s_tt[rr][zz])) *
                         C.inv_r_int[i];
            float a = C.ar_int[i];
            if (a != 0.f) {
                float q = C.br_int[i] * q0[p] + a * d_trr;
                S.psi_w[0][c] = q;
                d_trr += q;
            }
            a = C.az_int[j];
            if (a != 0.f) {
                float q = C.bz_int[j] * q1[p] + a * d_trz;
                S.psi_w[1][c] = q;
                d_trz += q;
            }
            S.vr[c] = vr0[p] + g.dt * br[p] * (d_trr + d_trz + hoop);
        }
        float d_trz = d4(s_rz[rr + 1][zz], s_rz[rr][zz], s_rz[rr + 2][zz], s_rz[rr - 1][zz]) * g.inv_dr;
        float d_tzz = d4(s_zz[rr][zz + 1], s_zz[rr][zz], s_zz[rr][zz + 2], s_zz[rr][zz - 1]) * g.inv_dz;
        float hoop = 0.5f * (s_rz[rr][zz] + s_rz[rr + 1][zz]) * C.inv_r_half[i];
        float a = C.ar_half[i];
        if (a != 0.f) {
            float q = C.br_half[i] * q2[p] + a * d_trz;
            S.psi_w[2][c] = q;
            d_trz += q;
        }
        a = C.az_half[j];
        if (a != 0.f) {
            float q = C.bz_half[j] * q3[p] + a * d_tzz;
            S.psi_w[3][c] = q;
            d_tzz += q;
        }
        S.vz[c] = vz0[p] + g.dt * bz[p] * (d_trz + d_tzz + hoop);
        if (hist0) {
            hist0[c] = vr0[p];
            hist0[g.nr * g.P + c] = vz0[p];
        }
    }
}

// Stress half-step of one tile: Eq. 2 lines 3-6 with the C-PML memories
// 4..7, source injection into the three normal stresses, pressure
// recording, and the store of v^{n+1/2} for the adjoint.  Own-node inputs
// are prefetched as in the velocity tile.
__device__ __forceinline__ void fwd_stress_tile(const WinK& g, const CoefK& C, const StateK& S,
                                                const SrcRecK& q, int n, bool record,
                                                float* hist, int i0, int j0, FwdSmem& sm)
{
    Tile &s_vr = sm.a, &s_vz = sm.b;
    const int j = j0 + threadIdx.x, zz = threadIdx.x + kH;
    const bool jok = j < g.nz;
    float t_rr[2], t_tt[2], t_zz[2], t_rz[2], lm[2], mu[2], mh[2], q4[2], q5[2], q6[2], q7[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int i = i0 + threadIdx.y + 8 * p;
        t_rr[p] = t_tt[p] = t_zz[p] = t_rz[p] = lm[p] = mu[p] = mh[p] = 0.f;
        q4[p] = q5[p] = q6[p] = q7[p] = 0.f;
        if (jok && i < g.nr) {
            const int c = i * g.P + j;
            const size_t cg = (size_t)i * g.nzg + g.z0 + j;
            t_rr[p] = ldcg(S.trr + c);
            t_tt[p] = ldcg(S.ttt + c);
            t_zz[p] = ldcg(S.tzz + c);
            lm[p] = __ldg(C.lam + cg);
            mu[p] = __ldg(C.mu + cg);
            if (C.ar_half[i] != 0.f) q4[p] = ldcg(S.psi[4] + c);
            if (C.az_int[j] != 0.f) q5[p] = ldcg(S.psi[5] + c);
            if (i >= 1) {
                t_rz[p] = ldcg(S.trz + c);
                mh[p] = muh_at(C, g, i, j);
                if (C.az_half[j] != 0.f) q6[p] = ldcg(S.psi[6] + c);
                if (C.ar_int[i] != 0.f) q7[p] = ldcg(S.psi[7] + c);
            }
        }
    }
    __syncthreads();
    stage<ODD>(s_vr, S.vr, i0, j0, g);
    stage<EVEN>(s_vz, S.vz, i0, j0, g);
    __syncthreads();
    if (!jok) return;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int i = i0 + threadIdx.y + 8 * p, rr = threadIdx.y + 8 * p + kH;
        if (i >= g.nr) break;
        const int c = i * g.P + j;
        float d_vr = d4(s_vr[rr + 1][zz], s_vr[rr][zz], s_vr[rr + 2][zz], s_vr[rr - 1][zz]) * g.inv_dr;
        float vr_r = 0.5f * (s_vr[rr][zz] + s_vr[rr + 1][zz]) * C.inv_r_half[i];
        float d_vz = d4(s_vz[rr][zz], s_vz[rr][zz - 1], s_vz[rr][zz + 1], s_vz[rr][zz - 2]) * g.inv_dz;
        float a = C.ar_half[i];
        if (a != 0.f) {
            float w = C.br_half[i] * q4[p] + a * d_vr;
            S.psi_w[4][c] = w;
            d_vr += w;
        }
        a = C.az_int[j];
        if (a != 0.f) {
            float w = C.bz_int[j] * q5[p] + a * d_vz;
            S.psi_w[5][c] = w;
            d_vz += w;
        }
        const float lam = lm[p];
        const float l2m = lam + 2.f * mu[p];
        float trr = t_rr[p] + g.dt * (l2m * d_vr + lam * (vr_r + d_vz));
        float ttt = t_tt[p] + g.dt * (l2m * vr_r + lam * (d_vr + d_vz));
        float tzz = t_zz[p] + g.dt * (l2m * d_vz + lam * (d_vr + vr_r));
        if (c == q.src_c) {
            float inj = q.src_scale * q.wavelet[n];
            trr += inj;
            ttt += inj;
            tzz += inj;
        }
        S.trr[c] = trr;
        S.ttt[c] = ttt;
        S.tzz[c] = tzz;
        if (i == 0 && record) {
            int k = q.recmap[j];
            if (k >= 0) q.seis[(size_t)k * q.nt + n] = (trr + ttt + tzz) * (1.f / 3.f);
        }
        if (i >= 1) {
            float d_vrz = d4(s_vr[rr][zz + 1], s_vr[rr][zz], s_vr[rr][zz + 2], s_vr[rr][zz - 1]) *
                          g.inv_dz;
            float d_vzr = d4(s_vz[rr][zz], s_vz[rr - 1][zz], s_vz[rr + 1][zz], s_vz[rr - 2][zz]) *
                          g.inv_dr;
            a = C.az_half[j];
            if (a != 0.f) {
                float w = C.bz_half[j] * q6[p] + a * d_vrz;
                S.psi_w[6][c] = w;
                d_vrz += w;
            }
            a = C.ar_int[i];
            if (a != 0.f) {
                float w = C.br_int[i] * q7[p] + a * d_vzr;
                S.psi_w[7][c] = w;
                d_vzr += w;
            }
            S.trz[c] = t_rz[p] + g.dt * mh[p] * (d_vrz + d_vzr);
        }
        if (hist) {
            hist[c] = s_vr[rr][zz];
            hist[g.nr * g.P + c] = s_vz[rr][zz];
        }
    }
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

// All blocks of a cooperative launch meet here; `epoch` counts the block's
// barriers (the same sequence in every block).  A block arrives with one
// release-acquire increment of a monotonic counter and waits, polling with
// acquire loads, until the counter reaches epoch * expected.  The wait is
// bounded twice, by the wall clock and by a poll count; when it runs out, or
// another block reports that it did, the function returns false in every
// thread of the block, the caller returns from the kernel, and the host reads
// the error flag.  Writes before the barrier are visible to ld.global.cg
// loads after it.
__device__ bool grid_barrier(const BarK& b, unsigned& epoch)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        ++epoch;
        const unsigned target = epoch * b.expected;
        unsigned old;
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(b.count) : "memory");
        int ok = 1;
        if (old + 1u < target) {
            const unsigned long long t0 = global_ns();
            const unsigned long long max_polls = b.timeout_ns / 64ull + 1024ull;
            unsigned long long polls = 0;
            volatile int* verr = b.err;
            for (;;) {
                unsigned cur;
                asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(b.count) : "memory");
                if (cur >= target) break;
                if (*verr) { ok = 0; break; }
                if (global_ns() - t0 > b.timeout_ns || ++polls > max_polls) {
                    atomicExch(b.err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (ok && *(volatile int*)b.err) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
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

struct AdjSmem {
    // staged: adjoint stresses, lambda, mu, mu_h, forward v^{n+1/2}
    Tile arr, att, azz, arz, lam, mu, muh, fvr, fvz;
    // transposed-stencil coefficients: on D_r v_r (x4), v_r/r (ytt), D_z v_z
    // (x5) at cells; on D_z v_r (x6) and D_r v_z (x7) at trz nodes.  The
    // velocity-step tile reuses x4..x7, ytt, arr as W_r, W_z, X0..X3.
    Tile x4, ytt, x5, x6, x7;
};

// stage a model field over the tile: cells (CELL) mirror evenly; trz nodes
// (harmonic mu) mirror about the axis row to row |i| with the window's own
// last-row rule
enum { CELL = 0, SHEAR = 1 };
template <int KIND>
__device__ __forceinline__ void stage_model(Tile& s, const float* __restrict__ f, const CoefK& C,
                                            int i0, int j0, const WinK& g)
{
    const int lane = threadIdx.x;
    for (int rr = threadIdx.y; rr < kSR; rr += 8) {
        int i = i0 - kH + rr;
        if (KIND == CELL) {
            if (i < 0) i = -1 - i;
        } else {
            if (i < 0) i = -i;
        }
        const bool live = i < g.nr && (KIND == CELL || i >= 1);
        for (int h = 0; h < 2; ++h) {
            const int zz = lane + 32 * h;
            if (zz >= kSZ) break;
            const int j = j0 - kH + zz;
            float v = 0.f;
            if (live && j >= 0 && j < g.nz)
                v = (KIND == CELL) ? __ldg(f + (size_t)i * g.nzg + g.z0 + j) : muh_at(C, g, i, j);
            s[rr][zz] = v;
        }
    }
}

// Own-node inputs of one row of the transposed stress step.
struct AdjStressOwn {
    float av_r, av_z, fvr_prev, fvz_prev;
    float2 g_lam, g_munn, g_murz, g_br, g_bz;
    float h_lam, h_munn, h_murz;
    float q4, q5, q6, q7;
};

__device__ __forceinline__ void adj_stress_own(const WinK& g, const CoefK& C, const StateK& S,
                                               const AdjK& q, const float* fprev, int i, int j,
                                               AdjStressOwn& o)
{
    const float2 z2 = make_float2(0.f, 0.f);
    o.av_r = o.av_z = o.fvr_prev = o.fvz_prev = 0.f;
    o.g_lam = o.g_munn = o.g_murz = o.g_br = o.g_bz = z2;
    o.h_lam = o.h_munn = o.h_murz = 0.f;
    o.q4 = o.q5 = o.q6 = o.q7 = 0.f;
    if (i >= g.nr || j >= g.nz) return;
    const int c = i * g.P + j;
    const int plane = g.nr * g.P;
    o.av_z = ldcg(S.vz + c);
    o.g_lam = __ldcg(q.G_lam + c);
    o.g_munn = __ldcg(q.G_munn + c);
    o.g_bz = __ldcg(q.G_bz + c);
    o.h_lam = ldcg(q.H_lam + c);
    o.h_munn = ldcg(q.H_munn + c);
    o.fvz_prev = __ldg(fprev + plane + c);
    if (C.ar_half[i] != 0.f) o.q4 = ldcg(S.psi[4] + c);
    if (C.az_int[j] != 0.f) o.q5 = ldcg(S.psi[5] + c);
    if (i >= 1) {
        o.av_r = ldcg(S.vr + c);
        o.g_murz = __ldcg(q.G_murz + c);
        o.g_br = __ldcg(q.G_br + c);
        o.h_murz = ldcg(q.H_murz + c);
        o.fvr_prev = __ldg(fprev + c);
        if (C.az_half[j] != 0.f) o.q6 = ldcg(S.psi[6] + c);
        if (C.ar_int[i] != 0.f) o.q7 = ldcg(S.psi[7] + c);
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
// fcur: v_r, v_z planes of v^{n+1/2}; fprev: those of v^{n-1/2}
__device__ __forceinline__ void adj_stress_tile(const WinK& g, const CoefK& C, const StateK& S,
                                                const AdjK& q, const float* fcur,
                                                const float* fprev, int i0, int j0, AdjSmem& sm)
{
    const float* fvr = fcur;
    const float* fvz = fcur + g.nr * g.P;
    const float dt = g.dt;
    const int j = j0 + threadIdx.x, zz = threadIdx.x + kH;
    AdjStressOwn own;
    adj_stress_own(g, C, S, q, fprev, i0 + threadIdx.y, j, own);
    __syncthreads();
    stage<EVEN>(sm.arr, S.trr, i0, j0, g);
    stage<EVEN>(sm.att, S.ttt, i0, j0, g);
    stage<EVEN>(sm.azz, S.tzz, i0, j0, g);
    stage<ODD>(sm.arz, S.trz, i0, j0, g);
    stage<ODD>(sm.fvr, fvr, i0, j0, g);
    stage<EVEN>(sm.fvz, fvz, i0, j0, g);
    stage_model<CELL>(sm.lam, C.lam, C, i0, j0, g);
    stage_model<CELL>(sm.mu, C.mu, C, i0, j0, g);
    stage_model<SHEAR>(sm.muh, nullptr, C, i0, j0, g);
    // adjoint memories read by the staged coefficients (inside the layers only)
    {
        const int lane = threadIdx.x;
        for (int rr = threadIdx.y; rr < kSR; rr += 8) {
            const int i = i0 - kH + rr;
            const int ic = i < 0 ? -1 - i : i;
            const bool row_cell = i < g.nr;
            const bool arh = row_cell && C.ar_half[ic] != 0.f;
            const bool ari = i >= 1 && i < g.nr && C.ar_int[i] != 0.f;
            for (int h = 0; h < 2; ++h) {
                const int zz2 = lane + 32 * h;
                if (zz2 >= kSZ) break;
                const int jj = j0 - kH + zz2;
                float p4 = 0.f, p5 = 0.f, p6 = 0.f, p7 = 0.f;
                if (jj >= 0 && jj < g.nz && row_cell) {
                    if (arh) p4 = ldcg(S.psi[4] + ic * g.P + jj);
                    if (C.az_int[jj] != 0.f) p5 = ldcg(S.psi[5] + ic * g.P + jj);
                    if (i >= 1 && C.az_half[jj] != 0.f) p6 = ldcg(S.psi[6] + i * g.P + jj);
                    if (ari) p7 = ldcg(S.psi[7] + i * g.P + jj);
                }
                sm.x4[rr][zz2] = p4;
                sm.x5[rr][zz2] = p5;
                sm.x6[rr][zz2] = p6;
                sm.x7[rr][zz2] = p7;
            }
        }
    }
    __syncthreads();
    // transposed-stencil coefficients over the staged region
    {
        const int lane = threadIdx.x;
        for (int rr = threadIdx.y; rr < kSR; rr += 8) {
            const int i = i0 - kH + rr;
            const int ic = i < 0 ? -1 - i : i;
            const bool row_cell = i < g.nr;
            const float arh = row_cell ? C.ar_half[ic] : 0.f;
            const float brh = row_cell ? C.br_half[ic] : 0.f;
            const float ari = (i >= 1 && i < g.nr) ? C.ar_int[i] : 0.f;
            const float bri = (i >= 1 && i < g.nr) ? C.br_int[i] : 0.f;
            for (int h = 0; h < 2; ++h) {
                const int zz2 = lane + 32 * h;
                if (zz2 >= kSZ) break;
                const int jj = j0 - kH + zz2;
                float x4 = 0.f, ytt = 0.f, x5 = 0.f, x6 = 0.f, x7 = 0.f;
                if (jj >= 0 && jj < g.nz && row_cell) {
                    const float lam = sm.lam[rr][zz2], l2m = lam + 2.f * sm.mu[rr][zz2];
                    const float arr = sm.arr[rr][zz2], att = sm.att[rr][zz2], azz = sm.azz[rr][zz2];
                    x4 = dt * (l2m * arr + lam * (att + azz));
                    ytt = dt * (l2m * att + lam * (arr + azz));
                    x5 = dt * (l2m * azz + lam * (arr + att));
                    if (arh != 0.f) x4 = x4 + arh * (x4 + brh * sm.x4[rr][zz2]);
                    const float azi = C.az_int[jj];
                    if (azi != 0.f) x5 = x5 + azi * (x5 + C.bz_int[jj] * sm.x5[rr][zz2]);
                    // trz node: the staged values are already odd about the axis
                    const float y = dt * sm.muh[rr][zz2] * sm.arz[rr][zz2];
                    x6 = y;
                    x7 = y;
                    if (i >= 1) {
                        const float azh = C.az_half[jj];
                        if (azh != 0.f) x6 = y + azh * (y + C.bz_half[jj] * sm.x6[rr][zz2]);
                        if (ari != 0.f) x7 = y + ari * (y + bri * sm.x7[rr][zz2]);
                    }
                }
                // each thread overwrites only the positions it read
                sm.x4[rr][zz2] = x4;
                sm.ytt[rr][zz2] = ytt;
                sm.x5[rr][zz2] = x5;
                sm.x6[rr][zz2] = x6;
                sm.x7[rr][zz2] = x7;
            }
        }
    }
    __syncthreads();

    if (j >= g.nz) return;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int i = i0 + threadIdx.y + 8 * p, rr = threadIdx.y + 8 * p + kH;
        if (i >= g.nr) break;
        const int c = i * g.P + j;
        if (p == 1) adj_stress_own(g, C, S, q, fprev, i, j, own);

        // ---- gradient correlation with the forward strains of v^{n+1/2}
        const float arr = sm.arr[rr][zz], att = sm.att[rr][zz], azz = sm.azz[rr][zz];
        float err = d4(sm.fvr[rr + 1][zz], sm.fvr[rr][zz], sm.fvr[rr + 2][zz], sm.fvr[rr - 1][zz]) *
                    g.inv_dr;
        float ett = 0.5f * (sm.fvr[rr][zz] + sm.fvr[rr + 1][zz]) * C.inv_r_half[i];
        float ezz = d4(sm.fvz[rr][zz], sm.fvz[rr][zz - 1], sm.fvz[rr][zz + 1], sm.fvz[rr][zz - 2]) *
                    g.inv_dz;
        float div = err + ett + ezz;
        q.G_lam[c] = kahan_step(own.g_lam, dt * div * (arr + att + azz));
        q.G_munn[c] = kahan_step(own.g_munn, 2.f * dt * (err * arr + ett * att + ezz * azz));
        q.H_lam[c] = own.h_lam + dt * div * div;
        q.H_munn[c] = own.h_munn + 4.f * dt * (err * err + ett * ett + ezz * ezz);

        // ---- transpose of the stress step into Av, and the density term
        {
            float sz = d4(sm.x5[rr][zz], sm.x5[rr][zz + 1], sm.x5[rr][zz - 1], sm.x5[rr][zz + 2]) * g.inv_dz;
            sz += d4(sm.x7[rr][zz], sm.x7[rr + 1][zz], sm.x7[rr - 1][zz], sm.x7[rr + 2][zz]) * g.inv_dr;
            const float av = own.av_z + sz;
            S.vz[c] = av;
            q.G_bz[c] = kahan_step(own.g_bz, (sm.fvz[rr][zz] - own.fvz_prev) * av);
        }
        const float lam = sm.lam[rr][zz], l2m = lam + 2.f * sm.mu[rr][zz];
        if (C.ar_half[i] != 0.f)
            S.psi_w[4][c] = dt * (l2m * arr + lam * (att + azz)) + C.br_half[i] * own.q4;
        if (C.az_int[j] != 0.f)
            S.psi_w[5][c] = dt * (l2m * azz + lam * (arr + att)) + C.bz_int[j] * own.q5;
        if (i >= 1) {
            float gam = d4(sm.fvr[rr][zz + 1], sm.fvr[rr][zz], sm.fvr[rr][zz + 2], sm.fvr[rr][zz - 1]) *
                            g.inv_dz +
                        d4(sm.fvz[rr][zz], sm.fvz[rr - 1][zz], sm.fvz[rr + 1][zz], sm.fvz[rr - 2][zz]) *
                            g.inv_dr;
            q.G_murz[c] = kahan_step(own.g_murz, dt * gam * sm.arz[rr][zz]);
            q.H_murz[c] = own.h_murz + dt * gam * gam;
            float sr = d4(sm.x4[rr - 1][zz], sm.x4[rr][zz], sm.x4[rr - 2][zz], sm.x4[rr + 1][zz]) * g.inv_dr;
            sr += 0.5f * (sm.ytt[rr - 1][zz] * C.inv_r_half[i - 1] + sm.ytt[rr][zz] * C.inv_r_half[i]);
            sr += d4(sm.x6[rr][zz - 1], sm.x6[rr][zz], sm.x6[rr][zz - 2], sm.x6[rr][zz + 1]) * g.inv_dz;
            const float av = own.av_r + sr;
            S.vr[c] = av;
            q.G_br[c] = kahan_step(own.g_br, (sm.fvr[rr][zz] - own.fvr_prev) * av);
            const float y = dt * sm.muh[rr][zz] * sm.arz[rr][zz];
            if (C.az_half[j] != 0.f) S.psi_w[6][c] = y + C.bz_half[j] * own.q6;
            if (C.ar_int[i] != 0.f) S.psi_w[7][c] = y + C.br_int[i] * own.q7;
        }
    }
}

// Transpose of the velocity step of one tile at reverse step n: S.{vr,vz}
// hold dJ/dv^{n+1/2}; S.{trr..trz} accumulate to dJ/dtau^n.  Then the
// residual of step n-1 is injected at the receivers (transpose of the
// recording).
__device__ __forceinline__ void adj_vel_tile(const WinK& g, const CoefK& C, const StateK& S,
                                             const AdjK& q, int n, int i0, int j0, AdjSmem& sm)
{
    // W = dt b Av at the velocity nodes (odd about the axis for v_r, even
    // for v_z), the coefficients on the four stretched derivatives, and the
    // old adjoint memories of the own nodes
    Tile &s_wr = sm.x4, &s_wz = sm.ytt, &s_x0 = sm.x5, &s_x1 = sm.x6, &s_x2 = sm.x7,
         &s_x3 = sm.arr, &s_p0 = sm.att, &s_p1 = sm.azz, &s_p2 = sm.arz, &s_p3 = sm.lam;
    const int j = j0 + threadIdx.x, zz = threadIdx.x + kH;
    const bool jok = j < g.nz;
    float o_rr[2], o_tt[2], o_zz[2], o_rz[2], r3[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int i = i0 + threadIdx.y + 8 * p;
        o_rr[p] = o_tt[p] = o_zz[p] = o_rz[p] = r3[p] = 0.f;
        if (jok && i < g.nr) {
            const int c = i * g.P + j;
            o_rr[p] = ldcg(S.trr + c);
            o_tt[p] = ldcg(S.ttt + c);
            o_zz[p] = ldcg(S.tzz + c);
            if (i >= 1) o_rz[p] = ldcg(S.trz + c);
            if (i == 0 && n > 0) {
                const int k = q.recmap[j];
                if (k >= 0) r3[p] = q.resid[(size_t)k * q.nt + (n - 1)] * (1.f / 3.f);
            }
        }
    }
    __syncthreads();
    {
        const int lane = threadIdx.x;
        for (int rr = threadIdx.y; rr < kSR; rr += 8) {
            const int i = i0 - kH + rr;
            const int ir = i < 0 ? -i : i;       // v_r node mirrored row
            const float sg = i < 0 ? -1.f : 1.f;
            const bool rlive = ir >= 1 && ir < g.nr;
            const int iz = i < 0 ? -1 - i : i;   // v_z node mirrored row
            const bool zlive = iz < g.nr;
            const float ari = rlive ? C.ar_int[ir] : 0.f, bri = rlive ? C.br_int[ir] : 0.f;
            const float arh = zlive ? C.ar_half[iz] : 0.f, brh = zlive ? C.br_half[iz] : 0.f;
            for (int h = 0; h < 2; ++h) {
                const int zz2 = lane + 32 * h;
                if (zz2 >= kSZ) break;
                const int jj = j0 - kH + zz2;
                float wr = 0.f, wz = 0.f, x0 = 0.f, x1 = 0.f, x2 = 0.f, x3 = 0.f;
                float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
                if (jj >= 0 && jj < g.nz) {
                    if (rlive) {
                        const int c = ir * g.P + jj;
                        const float w = g.dt * __ldg(C.bvr + (size_t)ir * g.nzg + g.z0 + jj) * ldcg(S.vr + c);
                        if (ari != 0.f) p0 = ldcg(S.psi[0] + c);
                        const float a = C.az_int[jj];
                        if (a != 0.f) p1 = ldcg(S.psi[1] + c);
                        x0 = (ari != 0.f) ? w + ari * (w + bri * p0) : w;
                        x1 = (a != 0.f) ? w + a * (w + C.bz_int[jj] * p1) : w;
                        wr = sg * w;
                        x0 *= sg;
                        x1 *= sg;
                    }
                    if (zlive) {
                        const int c = iz * g.P + jj;
                        const float w = g.dt * bvz_at(C, g, iz, jj) * ldcg(S.vz + c);
                        if (arh != 0.f) p2 = ldcg(S.psi[2] + c);
                        const float a = C.az_half[jj];
                        if (a != 0.f) p3 = ldcg(S.psi[3] + c);
                        x2 = (arh != 0.f) ? w + arh * (w + brh * p2) : w;
                        x3 = (a != 0.f) ? w + a * (w + C.bz_half[jj] * p3) : w;
                        wz = w;
                    }
                }
                s_wr[rr][zz2] = wr;
                s_wz[rr][zz2] = wz;
                s_x0[rr][zz2] = x0;
                s_x1[rr][zz2] = x1;
                s_x2[rr][zz2] = x2;
                s_x3[rr][zz2] = x3;
                s_p0[rr][zz2] = p0;
                s_p1[rr][zz2] = p1;
                s_p2[rr][zz2] = p2;
                s_p3[rr][zz2] = p3;
            }
        }
    }
    __syncthreads();

    if (!jok) return;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int i = i0 + threadIdx.y + 8 * p, rr = threadIdx.y + 8 * p + kH;
        if (i >= g.nr) break;
        const int c = i * g.P + j;
        // cell (i,j); inv_r_int[0] is 0 and W_r vanishes on the axis
        float hoop = 0.5f * (s_wr[rr][zz] * C.inv_r_int[i] +
                             s_wr[rr + 1][zz] * (i + 1 < g.nr ? C.inv_r_int[i + 1] : 0.f));
        float arr = d4(s_x0[rr][zz], s_x0[rr + 1][zz], s_x0[rr - 1][zz], s_x0[rr + 2][zz]) * g.inv_dr;
        float azz = d4(s_x3[rr][zz - 1], s_x3[rr][zz], s_x3[rr][zz - 2], s_x3[rr][zz + 1]) * g.inv_dz;
        S.trr[c] = o_rr[p] + arr + hoop + r3[p];
        S.ttt[c] = o_tt[p] - hoop + r3[p];
        S.tzz[c] = o_zz[p] + azz + r3[p];

        if (i >= 1) {
            float sr = d4(s_x1[rr][zz], s_x1[rr][zz + 1], s_x1[rr][zz - 1], s_x1[rr][zz + 2]) * g.inv_dz;
            sr += d4(s_x2[rr - 1][zz], s_x2[rr][zz], s_x2[rr - 2][zz], s_x2[rr + 1][zz]) * g.inv_dr;
            sr += 0.5f * (s_wz[rr - 1][zz] * C.inv_r_half[i - 1] + s_wz[rr][zz] * C.inv_r_half[i]);
            S.trz[c] = o_rz[p] + sr;
            const float w = s_wr[rr][zz];
            if (C.ar_int[i] != 0.f) S.psi_w[0][c] = w + C.br_int[i] * s_p0[rr][zz];
            if (C.az_int[j] != 0.f) S.psi_w[1][c] = w + C.bz_int[j] * s_p1[rr][zz];
        }
        {
            const float w = s_wz[rr][zz];
            if (C.ar_half[i] != 0.f) S.psi_w[2][c] = w + C.br_half[i] * s_p2[rr][zz];
            if (C.az_half[j] != 0.f) S.psi_w[3][c] = w + C.bz_half[j] * s_p3[rr][zz];
        }
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
    const int4* tiles;  // (shot within the table, i0, j0, 0)
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

template <int N>
__device__ __forceinline__ void run_fwd_vel(const RunK& r, const ShotTable<N>& T, int n, int t,
                                            FwdSmem& sm)
{
    const int4 tk = r.tiles[t];
    const ShotK& sh = shot_of(T, tk);
    float* h0 = (r.hist_n0 >= 0 && n == r.hist_n0) ? hist_slot(sh, 0) : nullptr;
    fwd_vel_tile(sh.g, sh.C, sh.Sf, h0, tk.y, tk.z, sm);
}

template <int N>
__device__ __forceinline__ void run_fwd_stress(const RunK& r, const ShotTable<N>& T, int n,
                                               int t, FwdSmem& sm)
{
    const int4 tk = r.tiles[t];
    const ShotK& sh = shot_of(T, tk);
    float* h = r.hist_n0 >= 0 ? hist_slot(sh, n - r.hist_n0 + 1) : nullptr;
    fwd_stress_tile(sh.g, sh.C, sh.Sf, sh.q, n, r.record != 0, h, tk.y, tk.z, sm);
}

template <int N>
__device__ __forceinline__ void run_adj_stress(const RunK& r, const ShotTable<N>& T, int n,
                                               int t, AdjSmem& sm)
{
    const int4 tk = r.tiles[t];
    const ShotK& sh = shot_of(T, tk);
    const int parity = (r.nt - 1 - n) & 1;
    adj_stress_tile(sh.g, sh.C, sh.Sa[parity], sh.a, hist_slot(sh, n - r.hist_n0 + 1),
                    hist_slot(sh, n - r.hist_n0), tk.y, tk.z, sm);
}

template <int N>
__device__ __forceinline__ void run_adj_vel(const RunK& r, const ShotTable<N>& T, int n, int t,
                                            AdjSmem& sm)
{
    const int4 tk = r.tiles[t];
    const ShotK& sh = shot_of(T, tk);
    const int parity = (r.nt - 1 - n) & 1;
    adj_vel_tile(sh.g, sh.C, sh.Sa[parity], sh.a, n, tk.y, tk.z, sm);
}

// one launch per half-step: one block per tile
template <int N>
__global__ void __launch_bounds__(kThreads) k_fwd_vel(RunK r, int n,
                                                      const __grid_constant__ ShotTable<N> T)
{
    __shared__ FwdSmem sm;
    pdl_wait();
    run_fwd_vel(r, T, n, blockIdx.x, sm);
    pdl_launch_dependents();
}

template <int N>
__global__ void __launch_bounds__(kThreads) k_fwd_stress(RunK r, int n,
                                                         const __grid_constant__ ShotTable<N> T)
{
    __shared__ FwdSmem sm;
    pdl_wait();
    run_fwd_stress(r, T, n, blockIdx.x, sm);
    pdl_launch_dependents();
}

template <int N>
__global__ void __launch_bounds__(kThreads) k_adj_stress(RunK r, int n,
                                                         const __grid_constant__ ShotTable<N> T)
{
    __shared__ AdjSmem sm;
    pdl_wait();
    run_adj_stress(r, T, n, blockIdx.x, sm);
    pdl_launch_dependents();
}

template <int N>
__global__ void __launch_bounds__(kThreads) k_adj_vel(RunK r, int n,
                                                      const __grid_constant__ ShotTable<N> T)
{
    __shared__ AdjSmem sm;
    pdl_wait();
    run_adj_vel(r, T, n, blockIdx.x, sm);
    pdl_launch_dependents();
}

// every step n0 .. n1-1 of every shot of the table in one cooperative launch
template <int N>
__global__ void __launch_bounds__(kThreads, 5) k_fwd_persist(RunK r, BarK b,
                                                             const __grid_constant__ ShotTable<N> T)
{
    __shared__ FwdSmem sm;
    unsigned epoch = 0;
    for (int n = r.n0; n < r.n1; ++n) {
        for (int t = blockIdx.x; t < r.ntiles; t += gridDim.x) run_fwd_vel(r, T, n, t, sm);
        if (!grid_barrier(b, epoch)) return;
        for (int t = blockIdx.x; t < r.ntiles; t += gridDim.x) run_fwd_stress(r, T, n, t, sm);
        if (!grid_barrier(b, epoch)) return;
    }
}

// reverse steps n1-1 down to n0 of every shot of the table in one cooperative launch
template <int N>
__global__ void __launch_bounds__(kThreads, 5) k_adj_persist(RunK r, BarK b,
                                                             const __grid_constant__ ShotTable<N> T)
{
    __shared__ AdjSmem sm;
    unsigned epoch = 0;
    for (int n = r.n1 - 1; n >= r.n0; --n) {
        for (int t = blockIdx.x; t < r.ntiles; t += gridDim.x) run_adj_stress(r, T, n, t, sm);
        if (!grid_barrier(b, epoch)) return;
        for (int t = blockIdx.x; t < r.ntiles; t += gridDim.x) run_adj_vel(r, T, n, t, sm);
        if (!grid_barrier(b, epoch)) return;
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
