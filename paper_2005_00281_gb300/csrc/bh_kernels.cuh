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

__device__ __forceinline__ void kahan_add(float2* __restrict__ acc, size_t k, float x)
{
    float2 s = acc[k];
    float y = __fsub_rn(x, s.y);
    float t = __fadd_rn(s.x, y);
    s.y = __fsub_rn(__fsub_rn(t, s.x), y);
    s.x = t;
    acc[k] = s;
}

// ------------------------------------------------------------- tiling
//
// Every stepping kernel works on a tile of TR x TZ nodes (16 rows of r by 32
// columns of z; 256 threads, each thread two rows 8 apart so that a warp
// always covers 32 consecutive z) and first stages what its stencils read
// from the tile plus a 2-node halo into shared memory, with the axis mirror
// and the zero edges already applied.  The adjoint kernels then build the
// transposed-stencil coefficients once per staged node.
constexpr int kTZ = 32, kTR = 16, kH = 2;
constexpr int kSZ = kTZ + 2 * kH, kSR = kTR + 2 * kH, kNS = kSZ * kSR;
constexpr int kThreads = 256;

// Programmatic dependent launch: a kernel may be scheduled while its
// predecessor drains; it must wait here before touching the predecessor's
// outputs.  No-op when launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// model value at window cell (i, j), i and j in range
__device__ __forceinline__ float ldm(const float* __restrict__ f, int i, int j, const WinK& g)
{
    return f[(size_t)i * g.nzg + g.z0 + j];
}

// ------------------------------------------------------- forward: Eq. 2

// Velocity half-step: Eq. 2 lines 1-2 with the C-PML memories 0..3.
__global__ void __launch_bounds__(kThreads) k_fwd_vel(WinK g, CoefK C, StateK S)
{
    __shared__ float s_rr[kSR][kSZ], s_tt[kSR][kSZ], s_rz[kSR][kSZ], s_zz[kSR][kSZ];
    pdl_wait();
    const int j0 = blockIdx.x * kTZ, i0 = blockIdx.y * kTR;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int k = tid; k < kNS; k += kThreads) {
        const int rr = k / kSZ, zz = k - rr * kSZ;
        const int i = i0 - kH + rr, j = j0 - kH + zz;
        s_rr[rr][zz] = ld_h(S.trr, i, j, g);
        s_tt[rr][zz] = ld_h(S.ttt, i, j, g);
        s_rz[rr][zz] = ld_i(S.trz, i, j, g);
        s_zz[rr][zz] = ld_h(S.tzz, i, j, g);
    }
    __syncthreads();
    pdl_launch_dependents();
    const int j = j0 + threadIdx.x, zz = threadIdx.x + kH;
    if (j >= g.nz) return;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int i = i0 + threadIdx.y + 8 * p, rr = threadIdx.y + 8 * p + kH;
        if (i >= g.nr) break;
        const size_t c = (size_t)i * g.P + j;
        const size_t cg = (size_t)i * g.nzg + g.z0 + j;
        if (i >= 1) {
            float d_trr = d4(s_rr[rr][zz], s_rr[rr - 1][zz], s_rr[rr + 1][zz], s_rr[rr - 2][zz]) *
                          g.inv_dr;
            float d_trz = d4(s_rz[rr][zz], s_rz[rr][zz - 1], s_rz[rr][zz + 1], s_rz[rr][zz - 2]) *
                          g.inv_dz;
            float hoop = 0.5f * ((s_rr[rr - 1][zz] - s_tt[rr - 1][zz]) + (s_rr[rr][zz] - s_tt[rr][zz])) *
                         C.inv_r_int[i];
            float a = C.ar_int[i];
            if (a != 0.f) {
                float q = C.br_int[i] * S.psi[0][c] + a * d_trr;
                S.psi_w[0][c] = q;
                d_trr += q;
            }
            a = C.az_int[j];
            if (a != 0.f) {
                float q = C.bz_int[j] * S.psi[1][c] + a * d_trz;
                S.psi_w[1][c] = q;
                d_trz += q;
            }
            S.vr[c] += g.dt * C.bvr[cg] * (d_trr + d_trz + hoop);
        }
        float d_trz = d4(s_rz[rr + 1][zz], s_rz[rr][zz], s_rz[rr + 2][zz], s_rz[rr - 1][zz]) * g.inv_dr;
        float d_tzz = d4(s_zz[rr][zz + 1], s_zz[rr][zz], s_zz[rr][zz + 2], s_zz[rr][zz - 1]) * g.inv_dz;
        float hoop = 0.5f * (s_rz[rr][zz] + s_rz[rr + 1][zz]) * C.inv_r_half[i];
        float a = C.ar_half[i];
        if (a != 0.f) {
            float q = C.br_half[i] * S.psi[2][c] + a * d_trz;
            S.psi_w[2][c] = q;
            d_trz += q;
        }
        a = C.az_half[j];
        if (a != 0.f) {
            float q = C.bz_half[j] * S.psi[3][c] + a * d_tzz;
            S.psi_w[3][c] = q;
            d_tzz += q;
        }
        S.vz[c] += g.dt * bvz_at(C, g, i, j) * (d_trz + d_tzz + hoop);
    }
}

struct SrcRecK {
    int src_c;            // window state index of the source cell
    float src_scale;      // dt / V
    const float* wavelet; // [nt]
    const int* recmap;    // [nz]: receiver number of cell (0, j) or -1
    float* seis;          // [nrec_max][nt] of this shot
    int nt, n;
    float* hist;          // [nt][2][nr*P] or nullptr
};

// Stress half-step: Eq. 2 lines 3-6 with the C-PML memories 4..7, source
// injection into the three normal stresses, pressure recording, and the
// store of v^{n+1/2} for the adjoint.
__global__ void __launch_bounds__(kThreads) k_fwd_stress(WinK g, CoefK C, StateK S, SrcRecK q)
{
    __shared__ float s_vr[kSR][kSZ], s_vz[kSR][kSZ];
    pdl_wait();
    const int j0 = blockIdx.x * kTZ, i0 = blockIdx.y * kTR;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int k = tid; k < kNS; k += kThreads) {
        const int rr = k / kSZ, zz = k - rr * kSZ;
        const int i = i0 - kH + rr, j = j0 - kH + zz;
        s_vr[rr][zz] = ld_i(S.vr, i, j, g);
        s_vz[rr][zz] = ld_h(S.vz, i, j, g);
    }
    __syncthreads();
    pdl_launch_dependents();
    const int j = j0 + threadIdx.x, zz = threadIdx.x + kH;
    if (j >= g.nz) return;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int i = i0 + threadIdx.y + 8 * p, rr = threadIdx.y + 8 * p + kH;
        if (i >= g.nr) break;
        const size_t c = (size_t)i * g.P + j;
        const size_t cg = (size_t)i * g.nzg + g.z0 + j;
        float d_vr = d4(s_vr[rr + 1][zz], s_vr[rr][zz], s_vr[rr + 2][zz], s_vr[rr - 1][zz]) * g.inv_dr;
        float vr_r = 0.5f * (s_vr[rr][zz] + s_vr[rr + 1][zz]) * C.inv_r_half[i];
        float d_vz = d4(s_vz[rr][zz], s_vz[rr][zz - 1], s_vz[rr][zz + 1], s_vz[rr][zz - 2]) * g.inv_dz;
        float a = C.ar_half[i];
        if (a != 0.f) {
            float w = C.br_half[i] * S.psi[4][c] + a * d_vr;
            S.psi_w[4][c] = w;
            d_vr += w;
        }
        a = C.az_int[j];
        if (a != 0.f) {
            float w = C.bz_int[j] * S.psi[5][c] + a * d_vz;
            S.psi_w[5][c] = w;
            d_vz += w;
        }
        const float lam = C.lam[cg];
        const float l2m = lam + 2.f * C.mu[cg];
        float trr = S.trr[c] + g.dt * (l2m * d_vr + lam * (vr_r + d_vz));
        float ttt = S.ttt[c] + g.dt * (l2m * vr_r + lam * (d_vr + d_vz));
        float tzz = S.tzz[c] + g.dt * (l2m * d_vz + lam * (d_vr + vr_r));
        if ((int)c == q.src_c) {
            float inj = q.src_scale * q.wavelet[q.n];
            trr += inj;
            ttt += inj;
            tzz += inj;
        }
        S.trr[c] = trr;
        S.ttt[c] = ttt;
        S.tzz[c] = tzz;
        if (i == 0) {
            int k = q.recmap[j];
            if (k >= 0) q.seis[(size_t)k * q.nt + q.n] = (trr + ttt + tzz) * (1.f / 3.f);
        }
        if (i >= 1) {
            float d_vrz = d4(s_vr[rr][zz + 1], s_vr[rr][zz], s_vr[rr][zz + 2], s_vr[rr][zz - 1]) *
                          g.inv_dz;
            float d_vzr = d4(s_vz[rr][zz], s_vz[rr - 1][zz], s_vz[rr + 1][zz], s_vz[rr - 2][zz]) *
                          g.inv_dr;
            a = C.az_half[j];
            if (a != 0.f) {
                float w = C.bz_half[j] * S.psi[6][c] + a * d_vrz;
                S.psi_w[6][c] = w;
                d_vrz += w;
            }
            a = C.ar_int[i];
            if (a != 0.f) {
                float w = C.br_int[i] * S.psi[7][c] + a * d_vzr;
                S.psi_w[7][c] = w;
                d_vzr += w;
            }
            S.trz[c] += g.dt * muh_at(C, g, i, j) * (d_vrz + d_vzr);
        }
        if (q.hist) {
            float* h = q.hist + (size_t)q.n * 2 * g.nr * g.P;
            h[c] = s_vr[rr][zz];
            h[(size_t)g.nr * g.P + c] = s_vz[rr][zz];
        }
    }
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
    int nt, n;            // reverse step being processed
    const float* hist;    // [nt][2][nr*P]: v^{n+1/2}
    float2 *G_lam, *G_munn, *G_murz, *G_br, *G_bz;  // Kahan pairs [nr*P]
    float *H_lam, *H_munn, *H_murz;                 // [nr*P]
};

// Transpose of the stress step at reverse step n, fused with the gradient
// correlations (Eq. 7, Eq. 8, and the density term).  S.{trr..trz} hold
// dJ/dtau^{n+1}; S.{vr,vz} accumulate to dJ/dv^{n+1/2}; psi[4..7] are the
// adjoint memories read side, psi_w[4..7] the write side.
__global__ void __launch_bounds__(kThreads) k_adj_stress(WinK g, CoefK C, StateK S, AdjK q)
{
    // staged inputs: adjoint stresses, lambda, mu, mu_h, forward v^{n+1/2}
    __shared__ float s_arr[kSR][kSZ], s_att[kSR][kSZ], s_azz[kSR][kSZ], s_arz[kSR][kSZ];
    __shared__ float s_lam[kSR][kSZ], s_mu[kSR][kSZ], s_muh[kSR][kSZ];
    __shared__ float s_fvr[kSR][kSZ], s_fvz[kSR][kSZ];
    // transposed-stencil coefficients: on D_r v_r (x4), v_r/r (ytt), D_z v_z
    // (x5) at cells; on D_z v_r (x6) and D_r v_z (x7) at trz nodes
    __shared__ float s_x4[kSR][kSZ], s_ytt[kSR][kSZ], s_x5[kSR][kSZ], s_x6[kSR][kSZ],
        s_x7[kSR][kSZ];
    pdl_wait();
    const int j0 = blockIdx.x * kTZ, i0 = blockIdx.y * kTR;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const float* fvr = q.hist + (size_t)q.n * 2 * g.nr * g.P;
    const float* fvz = fvr + (size_t)g.nr * g.P;
    const float dt = g.dt;

    for (int k = tid; k < kNS; k += kThreads) {
        const int rr = k / kSZ, zz = k - rr * kSZ;
        const int i = i0 - kH + rr, j = j0 - kH + zz;
        s_arr[rr][zz] = ld_h(S.trr, i, j, g);
        s_att[rr][zz] = ld_h(S.ttt, i, j, g);
        s_azz[rr][zz] = ld_h(S.tzz, i, j, g);
        s_arz[rr][zz] = ld_i(S.trz, i, j, g);
        s_fvr[rr][zz] = ld_i(fvr, i, j, g);
        s_fvz[rr][zz] = ld_h(fvz, i, j, g);
        float lam = 0.f, mu = 0.f, mh = 0.f;
        if (j >= 0 && j < g.nz) {
            const int ic = i < 0 ? -1 - i : i;  // cells: even about the axis
            const int it = i < 0 ? -i : i;      // trz nodes: mirror row of an integer node
            if (ic < g.nr) {
                lam = ldm(C.lam, ic, j, g);
                mu = ldm(C.mu, ic, j, g);
            }
            if (it >= 1 && it < g.nr) mh = muh_at(C, g, it, j);
        }
        s_lam[rr][zz] = lam;
        s_mu[rr][zz] = mu;
        s_muh[rr][zz] = mh;
    }
    __syncthreads();
    for (int k = tid; k < kNS; k += kThreads) {
        const int rr = k / kSZ, zz = k - rr * kSZ;
        const int i = i0 - kH + rr, j = j0 - kH + zz;
        float x4 = 0.f, ytt = 0.f, x5 = 0.f, x6 = 0.f, x7 = 0.f;
        if (j >= 0 && j < g.nz && i < g.nr) {
            const int ic = i < 0 ? -1 - i : i;
            const float lam = s_lam[rr][zz], l2m = lam + 2.f * s_mu[rr][zz];
            const float arr = s_arr[rr][zz], att = s_att[rr][zz], azz = s_azz[rr][zz];
            x4 = dt * (l2m * arr + lam * (att + azz));
            ytt = dt * (l2m * att + lam * (arr + azz));
            x5 = dt * (l2m * azz + lam * (arr + att));
            float a = C.ar_half[ic];
            if (a != 0.f) x4 = x4 + a * (x4 + C.br_half[ic] * S.psi[4][(size_t)ic * g.P + j]);
            a = C.az_int[j];
            if (a != 0.f) x5 = x5 + a * (x5 + C.bz_int[j] * S.psi[5][(size_t)ic * g.P + j]);
            // trz node: the staged values are already odd about the axis
            const float y = dt * s_muh[rr][zz] * s_arz[rr][zz];
            x6 = y;
            x7 = y;
            if (i >= 1) {
                a = C.az_half[j];
                if (a != 0.f) x6 = y + a * (y + C.bz_half[j] * S.psi[6][(size_t)i * g.P + j]);
                a = C.ar_int[i];
                if (a != 0.f) x7 = y + a * (y + C.br_int[i] * S.psi[7][(size_t)i * g.P + j]);
            }
        }
        s_x4[rr][zz] = x4;
        s_ytt[rr][zz] = ytt;
        s_x5[rr][zz] = x5;
        s_x6[rr][zz] = x6;
        s_x7[rr][zz] = x7;
    }
    __syncthreads();
    pdl_launch_dependents();

    const int j = j0 + threadIdx.x, zz = threadIdx.x + kH;
    if (j >= g.nz) return;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int i = i0 + threadIdx.y + 8 * p, rr = threadIdx.y + 8 * p + kH;
        if (i >= g.nr) break;
        const size_t c = (size_t)i * g.P + j;

        // ---- gradient correlation with the forward strains of v^{n+1/2}
        const float arr = s_arr[rr][zz], att = s_att[rr][zz], azz = s_azz[rr][zz];
        {
            float err = d4(s_fvr[rr + 1][zz], s_fvr[rr][zz], s_fvr[rr + 2][zz], s_fvr[rr - 1][zz]) *
                        g.inv_dr;
            float ett = 0.5f * (s_fvr[rr][zz] + s_fvr[rr + 1][zz]) * C.inv_r_half[i];
            float ezz = d4(s_fvz[rr][zz], s_fvz[rr][zz - 1], s_fvz[rr][zz + 1], s_fvz[rr][zz - 2]) *
                        g.inv_dz;
            float div = err + ett + ezz;
            kahan_add(q.G_lam, c, dt * div * (arr + att + azz));
            kahan_add(q.G_munn, c, 2.f * dt * (err * arr + ett * att + ezz * azz));
            q.H_lam[c] += dt * div * div;
            q.H_munn[c] += 4.f * dt * (err * err + ett * ett + ezz * ezz);
            if (i >= 1) {
                float gam = d4(s_fvr[rr][zz + 1], s_fvr[rr][zz], s_fvr[rr][zz + 2], s_fvr[rr][zz - 1]) *
                                g.inv_dz +
                            d4(s_fvz[rr][zz], s_fvz[rr - 1][zz], s_fvz[rr + 1][zz], s_fvz[rr - 2][zz]) *
                                g.inv_dr;
                kahan_add(q.G_murz, c, dt * gam * s_arz[rr][zz]);
                q.H_murz[c] += dt * gam * gam;
            }
        }

        // ---- transpose of the stress step into Av, and the density term
        if (i >= 1) {
            float s = d4(s_x4[rr - 1][zz], s_x4[rr][zz], s_x4[rr - 2][zz], s_x4[rr + 1][zz]) * g.inv_dr;
            s += 0.5f * (s_ytt[rr - 1][zz] * C.inv_r_half[i - 1] + s_ytt[rr][zz] * C.inv_r_half[i]);
            s += d4(s_x6[rr][zz - 1], s_x6[rr][zz], s_x6[rr][zz - 2], s_x6[rr][zz + 1]) * g.inv_dz;
            float av = S.vr[c] + s;
            S.vr[c] = av;
            float dv = s_fvr[rr][zz] - (q.n > 0 ? fvr[c - (size_t)2 * g.nr * g.P] : 0.f);
            kahan_add(q.G_br, c, dv * av);
        }
        {
            float s = d4(s_x5[rr][zz], s_x5[rr][zz + 1], s_x5[rr][zz - 1], s_x5[rr][zz + 2]) * g.inv_dz;
            s += d4(s_x7[rr][zz], s_x7[rr + 1][zz], s_x7[rr - 1][zz], s_x7[rr + 2][zz]) * g.inv_dr;
            float av = S.vz[c] + s;
            S.vz[c] = av;
            float dv = s_fvz[rr][zz] - (q.n > 0 ? fvz[c - (size_t)2 * g.nr * g.P] : 0.f);
            kahan_add(q.G_bz, c, dv * av);
        }

        // ---- adjoint memories of the stress step (own cell / own shear node)
        {
            const float lam = s_lam[rr][zz], l2m = lam + 2.f * s_mu[rr][zz];
            if (C.ar_half[i] != 0.f)
                S.psi_w[4][c] = dt * (l2m * arr + lam * (att + azz)) + C.br_half[i] * S.psi[4][c];
            if (C.az_int[j] != 0.f)
                S.psi_w[5][c] = dt * (l2m * azz + lam * (arr + att)) + C.bz_int[j] * S.psi[5][c];
            if (i >= 1) {
                const float y = dt * s_muh[rr][zz] * s_arz[rr][zz];
                if (C.az_half[j] != 0.f) S.psi_w[6][c] = y + C.bz_half[j] * S.psi[6][c];
                if (C.ar_int[i] != 0.f) S.psi_w[7][c] = y + C.br_int[i] * S.psi[7][c];
            }
        }
    }
}

// Transpose of the velocity step at reverse step n: S.{vr,vz} hold
// dJ/dv^{n+1/2}; S.{trr..trz} accumulate to dJ/dtau^n.  Then the residual
// of step n-1 is injected at the receivers (transpose of the recording).
__global__ void __launch_bounds__(kThreads) k_adj_vel(WinK g, CoefK C, StateK S, AdjK q)
{
    // W = dt b Av at the velocity nodes (odd about the axis for v_r, even
    // for v_z), and the coefficients on the four stretched derivatives
    __shared__ float s_wr[kSR][kSZ], s_wz[kSR][kSZ];
    __shared__ float s_x0[kSR][kSZ], s_x1[kSR][kSZ], s_x2[kSR][kSZ], s_x3[kSR][kSZ];
    pdl_wait();
    const int j0 = blockIdx.x * kTZ, i0 = blockIdx.y * kTR;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int k = tid; k < kNS; k += kThreads) {
        const int rr = k / kSZ, zz = k - rr * kSZ;
        const int i = i0 - kH + rr, j = j0 - kH + zz;
        float wr = 0.f, wz = 0.f, x0 = 0.f, x1 = 0.f, x2 = 0.f, x3 = 0.f;
        if (j >= 0 && j < g.nz) {
            // v_r node: odd extension, zero on the axis and beyond nr
            const int ir = i < 0 ? -i : i;
            if (ir >= 1 && ir < g.nr) {
                const float sg = i < 0 ? -1.f : 1.f;
                const size_t c = (size_t)ir * g.P + j;
                const float w = g.dt * ldm(C.bvr, ir, j, g) * S.vr[c];
                float a = C.ar_int[ir];
                x0 = (a != 0.f) ? w + a * (w + C.br_int[ir] * S.psi[0][c]) : w;
                a = C.az_int[j];
                x1 = (a != 0.f) ? w + a * (w + C.bz_int[j] * S.psi[1][c]) : w;
                wr = sg * w;
                x0 *= sg;
                x1 *= sg;
            }
            // v_z node: even extension, zero beyond nr
            const int iz = i < 0 ? -1 - i : i;
            if (iz < g.nr) {
                const size_t c = (size_t)iz * g.P + j;
                const float w = g.dt * bvz_at(C, g, iz, j) * S.vz[c];
                float a = C.ar_half[iz];
                x2 = (a != 0.f) ? w + a * (w + C.br_half[iz] * S.psi[2][c]) : w;
                a = C.az_half[j];
                x3 = (a != 0.f) ? w + a * (w + C.bz_half[j] * S.psi[3][c]) : w;
                wz = w;
            }
        }
        s_wr[rr][zz] = wr;
        s_wz[rr][zz] = wz;
        s_x0[rr][zz] = x0;
        s_x1[rr][zz] = x1;
        s_x2[rr][zz] = x2;
        s_x3[rr][zz] = x3;
    }
    __syncthreads();
    pdl_launch_dependents();

    const int j = j0 + threadIdx.x, zz = threadIdx.x + kH;
    if (j >= g.nz) return;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int i = i0 + threadIdx.y + 8 * p, rr = threadIdx.y + 8 * p + kH;
        if (i >= g.nr) break;
        const size_t c = (size_t)i * g.P + j;
        // cell (i,j); inv_r_int[0] is 0 and W_r vanishes on the axis
        float hoop = 0.5f * (s_wr[rr][zz] * C.inv_r_int[i] +
                             s_wr[rr + 1][zz] * (i + 1 < g.nr ? C.inv_r_int[i + 1] : 0.f));
        float arr = d4(s_x0[rr][zz], s_x0[rr + 1][zz], s_x0[rr - 1][zz], s_x0[rr + 2][zz]) * g.inv_dr;
        float azz = d4(s_x3[rr][zz - 1], s_x3[rr][zz], s_x3[rr][zz - 2], s_x3[rr][zz + 1]) * g.inv_dz;
        float trr = S.trr[c] + arr + hoop;
        float ttt = S.ttt[c] - hoop;
        float tzz = S.tzz[c] + azz;
        if (i == 0 && q.n > 0) {
            int k = q.recmap[j];
            if (k >= 0) {
                float r3 = q.resid[(size_t)k * q.nt + (q.n - 1)] * (1.f / 3.f);
                trr += r3;
                ttt += r3;
                tzz += r3;
            }
        }
        S.trr[c] = trr;
        S.ttt[c] = ttt;
        S.tzz[c] = tzz;

        if (i >= 1) {
            float s = d4(s_x1[rr][zz], s_x1[rr][zz + 1], s_x1[rr][zz - 1], s_x1[rr][zz + 2]) * g.inv_dz;
            s += d4(s_x2[rr - 1][zz], s_x2[rr][zz], s_x2[rr - 2][zz], s_x2[rr + 1][zz]) * g.inv_dr;
            s += 0.5f * (s_wz[rr - 1][zz] * C.inv_r_half[i - 1] + s_wz[rr][zz] * C.inv_r_half[i]);
            S.trz[c] += s;
            const float w = s_wr[rr][zz];
            if (C.ar_int[i] != 0.f) S.psi_w[0][c] = w + C.br_int[i] * S.psi[0][c];
            if (C.az_int[j] != 0.f) S.psi_w[1][c] = w + C.bz_int[j] * S.psi[1][c];
        }
        {
            const float w = s_wz[rr][zz];
            if (C.ar_half[i] != 0.f) S.psi_w[2][c] = w + C.br_half[i] * S.psi[2][c];
            if (C.az_half[j] != 0.f) S.psi_w[3][c] = w + C.bz_half[j] * S.psi[3][c];
        }
    }
}

// transpose of the recording at the last step: dp[nt-1]/3 into each normal stress
__global__ void k_adj_inject(WinK g, StateK S, AdjK q, int nrec)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.nz) return;
    int r = q.recmap[k];
    if (r < 0) return;
    float r3 = q.resid[(size_t)r * q.nt + q.n] * (1.f / 3.f);
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
__global__ void k_finalize(WinK g, CoefK C, AdjK q, FinK f)
{
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
    f.g_lam[cg] += gl;
    f.g_mu[cg] += gm;
    f.H_lam[cg] += hl;
    f.H_mu[cg] += hm;
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
        f.g_rho[cg] += -0.5 / (rho * rho) * gb;
    }
}

}  // namespace bh
