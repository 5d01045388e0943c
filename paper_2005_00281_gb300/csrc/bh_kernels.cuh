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

// ------------------------------------------------------- forward: Eq. 2

// Velocity half-step: Eq. 2 lines 1-2 with the C-PML memories 0..3.
__global__ void __launch_bounds__(256) k_fwd_vel(WinK g, CoefK C, StateK S)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nr || j >= g.nz) return;
    const size_t c = (size_t)i * g.P + j;
    const size_t cg = (size_t)i * g.nzg + g.z0 + j;
    if (i >= 1) {
        float d_trr = d4(ld_h(S.trr, i, j, g), ld_h(S.trr, i - 1, j, g), ld_h(S.trr, i + 1, j, g),
                         ld_h(S.trr, i - 2, j, g)) * g.inv_dr;
        float d_trz = d4(ld_i(S.trz, i, j, g), ld_i(S.trz, i, j - 1, g), ld_i(S.trz, i, j + 1, g),
                         ld_i(S.trz, i, j - 2, g)) * g.inv_dz;
        float hoop = 0.5f * ((S.trr[c - g.P] - S.ttt[c - g.P]) + (S.trr[c] - S.ttt[c])) *
                     C.inv_r_int[i];
        float a = C.ar_int[i];
        if (a != 0.f) {
            float p = C.br_int[i] * S.psi[0][c] + a * d_trr;
            S.psi_w[0][c] = p;
            d_trr += p;
        }
        a = C.az_int[j];
        if (a != 0.f) {
            float p = C.bz_int[j] * S.psi[1][c] + a * d_trz;
            S.psi_w[1][c] = p;
            d_trz += p;
        }
        S.vr[c] += g.dt * C.bvr[cg] * (d_trr + d_trz + hoop);
    }
    float d_trz = d4(ld_i(S.trz, i + 1, j, g), ld_i(S.trz, i, j, g), ld_i(S.trz, i + 2, j, g),
                     ld_i(S.trz, i - 1, j, g)) * g.inv_dr;
    float d_tzz = d4(ld_h(S.tzz, i, j + 1, g), ld_h(S.tzz, i, j, g), ld_h(S.tzz, i, j + 2, g),
                     ld_h(S.tzz, i, j - 1, g)) * g.inv_dz;
    float hoop = 0.5f * (ld_i(S.trz, i, j, g) + ld_i(S.trz, i + 1, j, g)) * C.inv_r_half[i];
    float a = C.ar_half[i];
    if (a != 0.f) {
        float p = C.br_half[i] * S.psi[2][c] + a * d_trz;
        S.psi_w[2][c] = p;
        d_trz += p;
    }
    a = C.az_half[j];
    if (a != 0.f) {
        float p = C.bz_half[j] * S.psi[3][c] + a * d_tzz;
        S.psi_w[3][c] = p;
        d_tzz += p;
    }
    S.vz[c] += g.dt * bvz_at(C, g, i, j) * (d_trz + d_tzz + hoop);
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
__global__ void __launch_bounds__(256) k_fwd_stress(WinK g, CoefK C, StateK S, SrcRecK q)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nr || j >= g.nz) return;
    const size_t c = (size_t)i * g.P + j;
    const size_t cg = (size_t)i * g.nzg + g.z0 + j;

    float d_vr = d4(ld_i(S.vr, i + 1, j, g), ld_i(S.vr, i, j, g), ld_i(S.vr, i + 2, j, g),
                    ld_i(S.vr, i - 1, j, g)) * g.inv_dr;
    float vr_r = 0.5f * (ld_i(S.vr, i, j, g) + ld_i(S.vr, i + 1, j, g)) * C.inv_r_half[i];
    float d_vz = d4(ld_h(S.vz, i, j, g), ld_h(S.vz, i, j - 1, g), ld_h(S.vz, i, j + 1, g),
                    ld_h(S.vz, i, j - 2, g)) * g.inv_dz;
    float a = C.ar_half[i];
    if (a != 0.f) {
        float p = C.br_half[i] * S.psi[4][c] + a * d_vr;
        S.psi_w[4][c] = p;
        d_vr += p;
    }
    a = C.az_int[j];
    if (a != 0.f) {
        float p = C.bz_int[j] * S.psi[5][c] + a * d_vz;
        S.psi_w[5][c] = p;
        d_vz += p;
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
        float d_vrz = d4(ld_i(S.vr, i, j + 1, g), ld_i(S.vr, i, j, g), ld_i(S.vr, i, j + 2, g),
                         ld_i(S.vr, i, j - 1, g)) * g.inv_dz;
        float d_vzr = d4(ld_h(S.vz, i, j, g), ld_h(S.vz, i - 1, j, g), ld_h(S.vz, i + 1, j, g),
                         ld_h(S.vz, i - 2, j, g)) * g.inv_dr;
        a = C.az_half[j];
        if (a != 0.f) {
            float p = C.bz_half[j] * S.psi[6][c] + a * d_vrz;
            S.psi_w[6][c] = p;
            d_vrz += p;
        }
        a = C.ar_int[i];
        if (a != 0.f) {
            float p = C.br_int[i] * S.psi[7][c] + a * d_vzr;
            S.psi_w[7][c] = p;
            d_vzr += p;
        }
        S.trz[c] += g.dt * muh_at(C, g, i, j) * (d_vrz + d_vzr);
    }
    if (q.hist) {
        float* h = q.hist + (size_t)q.n * 2 * g.nr * g.P;
        h[c] = S.vr[c];
        h[(size_t)g.nr * g.P + c] = S.vz[c];
    }
}

// ------------------------------------------ adjoint: transpose of Eq. 2

struct AdjK {
    const float* resid;   // [nrec_max][nt] of this shot
    const int* recmap;    // [nz]
    int nt, n;            // reverse step being processed
    const float* hist;    // [nt][2][nr*P]: v^{n+1/2}
    float2 *G_lam, *G_munn, *G_murz, *G_br, *G_bz;  // Kahan pairs [nr*P]
    float *H_lam, *H_munn, *H_murz;                 // [nr*P]
};

// Adjoint of the stress-step quantities at a cell: the coefficient that the
// transposed stencil applies to D_r v_r (x_rr), to v_r/r (y_tt) and to
// D_z v_z (x_zz).  Cells outside the window give zero.
__device__ __forceinline__ float adj_x_rr(const WinK& g, const CoefK& C, const StateK& S,
                                          int i, int j)
{
    if (j < 0 || j >= g.nz || i >= g.nr) return 0.f;
    if (i < 0) i = -1 - i;  // even extension about the axis
    const size_t c = (size_t)i * g.P + j;
    const size_t cg = (size_t)i * g.nzg + g.z0 + j;
    const float lam = C.lam[cg], l2m = lam + 2.f * C.mu[cg];
    float y = g.dt * (l2m * S.trr[c] + lam * (S.ttt[c] + S.tzz[c]));
    float a = C.ar_half[i];
    if (a != 0.f) y = y + a * (y + C.br_half[i] * S.psi[4][c]);
    return y;
}

__device__ __forceinline__ float adj_y_tt(const WinK& g, const CoefK& C, const StateK& S,
                                          int i, int j)
{
    const size_t c = (size_t)i * g.P + j;
    const size_t cg = (size_t)i * g.nzg + g.z0 + j;
    const float lam = C.lam[cg], l2m = lam + 2.f * C.mu[cg];
    return g.dt * (l2m * S.ttt[c] + lam * (S.trr[c] + S.tzz[c]));
}

__device__ __forceinline__ float adj_x_zz(const WinK& g, const CoefK& C, const StateK& S,
                                          int i, int j)
{
    if (j < 0 || j >= g.nz) return 0.f;
    const size_t c = (size_t)i * g.P + j;
    const size_t cg = (size_t)i * g.nzg + g.z0 + j;
    const float lam = C.lam[cg], l2m = lam + 2.f * C.mu[cg];
    float y = g.dt * (l2m * S.tzz[c] + lam * (S.trr[c] + S.ttt[c]));
    float a = C.az_int[j];
    if (a != 0.f) y = y + a * (y + C.bz_int[j] * S.psi[5][c]);
    return y;
}

// shear node: coefficient on D_z v_r (x6, axial layer) and on D_r v_z (x7,
// radial layer); odd extension about the axis, zero outside
__device__ __forceinline__ float adj_x_rz_z(const WinK& g, const CoefK& C, const StateK& S,
                                            int i, int j)
{
    if (j < 0 || j >= g.nz) return 0.f;
    const size_t c = (size_t)i * g.P + j;
    float y = g.dt * muh_at(C, g, i, j) * S.trz[c];
    float a = C.az_half[j];
    if (a != 0.f) y = y + a * (y + C.bz_half[j] * S.psi[6][c]);
    return y;
}

__device__ __forceinline__ float adj_x_rz_r(const WinK& g, const CoefK& C, const StateK& S,
                                            int i, int j)
{
    float s = 1.f;
    if (i < 0) { i = -i; s = -1.f; }
    if (i == 0 || i >= g.nr) return 0.f;
    const size_t c = (size_t)i * g.P + j;
    float y = g.dt * muh_at(C, g, i, j) * S.trz[c];
    float a = C.ar_int[i];
    if (a != 0.f) y = y + a * (y + C.br_int[i] * S.psi[7][c]);
    return s * y;
}

// Transpose of the stress step at reverse step n, fused with the gradient
// correlations (Eq. 7, Eq. 8, and the density term).  S.{trr..trz} hold
// dJ/dtau^{n+1}; S.{vr,vz} accumulate to dJ/dv^{n+1/2}; psi[4..7] are the
// adjoint memories read side, psi_w[4..7] the write side.
__global__ void __launch_bounds__(256) k_adj_stress(WinK g, CoefK C, StateK S, AdjK q)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nr || j >= g.nz) return;
    const size_t c = (size_t)i * g.P + j;
    const float dt = g.dt;

    // ---- gradient correlation with the forward strains of v^{n+1/2}
    const float* fvr = q.hist + (size_t)q.n * 2 * g.nr * g.P;
    const float* fvz = fvr + (size_t)g.nr * g.P;
    {
        float err = d4(ld_i(fvr, i + 1, j, g), ld_i(fvr, i, j, g), ld_i(fvr, i + 2, j, g),
                       ld_i(fvr, i - 1, j, g)) * g.inv_dr;
        float ett = 0.5f * (ld_i(fvr, i, j, g) + ld_i(fvr, i + 1, j, g)) * C.inv_r_half[i];
        float ezz = d4(ld_h(fvz, i, j, g), ld_h(fvz, i, j - 1, g), ld_h(fvz, i, j + 1, g),
                       ld_h(fvz, i, j - 2, g)) * g.inv_dz;
        float arr = S.trr[c], att = S.ttt[c], azz = S.tzz[c];
        float div = err + ett + ezz;
        kahan_add(q.G_lam, c, dt * div * (arr + att + azz));
        kahan_add(q.G_munn, c, 2.f * dt * (err * arr + ett * att + ezz * azz));
        q.H_lam[c] += dt * div * div;
        q.H_munn[c] += 4.f * dt * (err * err + ett * ett + ezz * ezz);
        if (i >= 1) {
            float gam = d4(ld_i(fvr, i, j + 1, g), ld_i(fvr, i, j, g), ld_i(fvr, i, j + 2, g),
                           ld_i(fvr, i, j - 1, g)) * g.inv_dz +
                        d4(ld_h(fvz, i, j, g), ld_h(fvz, i - 1, j, g), ld_h(fvz, i + 1, j, g),
                           ld_h(fvz, i - 2, j, g)) * g.inv_dr;
            kahan_add(q.G_murz, c, dt * gam * S.trz[c]);
            q.H_murz[c] += dt * gam * gam;
        }
    }

    // ---- transpose of the stress step into Av
    if (i >= 1) {
        float s = d4(adj_x_rr(g, C, S, i - 1, j), adj_x_rr(g, C, S, i, j),
                     adj_x_rr(g, C, S, i - 2, j), adj_x_rr(g, C, S, i + 1, j)) * g.inv_dr;
        s += 0.5f * (adj_y_tt(g, C, S, i - 1, j) * C.inv_r_half[i - 1] +
                     adj_y_tt(g, C, S, i, j) * C.inv_r_half[i]);
        s += d4(adj_x_rz_z(g, C, S, i, j - 1), adj_x_rz_z(g, C, S, i, j),
                adj_x_rz_z(g, C, S, i, j - 2), adj_x_rz_z(g, C, S, i, j + 1)) * g.inv_dz;
        float av = S.vr[c] + s;
        S.vr[c] = av;
        float dv = fvr[c] - (q.n > 0 ? fvr[c - (size_t)2 * g.nr * g.P] : 0.f);
        kahan_add(q.G_br, c, dv * av);
    }
    {
        float s = d4(adj_x_zz(g, C, S, i, j), adj_x_zz(g, C, S, i, j + 1),
                     adj_x_zz(g, C, S, i, j - 1), adj_x_zz(g, C, S, i, j + 2)) * g.inv_dz;
        s += d4(adj_x_rz_r(g, C, S, i, j), adj_x_rz_r(g, C, S, i + 1, j),
                adj_x_rz_r(g, C, S, i - 1, j), adj_x_rz_r(g, C, S, i + 2, j)) * g.inv_dr;
        float av = S.vz[c] + s;
        S.vz[c] = av;
        float dv = fvz[c] - (q.n > 0 ? fvz[c - (size_t)2 * g.nr * g.P] : 0.f);
        kahan_add(q.G_bz, c, dv * av);
    }

    // ---- adjoint memories of the stress step (own cell / own shear node)
    {
        const size_t cg = (size_t)i * g.nzg + g.z0 + j;
        const float lam = C.lam[cg], l2m = lam + 2.f * C.mu[cg];
        float a = C.ar_half[i];
        if (a != 0.f)
            S.psi_w[4][c] = dt * (l2m * S.trr[c] + lam * (S.ttt[c] + S.tzz[c])) +
                            C.br_half[i] * S.psi[4][c];
        a = C.az_int[j];
        if (a != 0.f)
            S.psi_w[5][c] = dt * (l2m * S.tzz[c] + lam * (S.trr[c] + S.ttt[c])) +
                            C.bz_int[j] * S.psi[5][c];
        if (i >= 1) {
            float y = dt * muh_at(C, g, i, j) * S.trz[c];
            a = C.az_half[j];
            if (a != 0.f) S.psi_w[6][c] = y + C.bz_half[j] * S.psi[6][c];
            a = C.ar_int[i];
            if (a != 0.f) S.psi_w[7][c] = y + C.br_int[i] * S.psi[7][c];
        }
    }
}

// velocity-node adjoint weights W = dt b Av, and the coefficients applied
// to the four stretched derivatives of the velocity step
__device__ __forceinline__ float adj_w_r(const WinK& g, const CoefK& C, const StateK& S,
                                         int i, int j)
{
    if (i <= 0 || i >= g.nr || j < 0 || j >= g.nz) return 0.f;
    const size_t c = (size_t)i * g.P + j;
    return g.dt * C.bvr[(size_t)i * g.nzg + g.z0 + j] * S.vr[c];
}

__device__ __forceinline__ float adj_w_z(const WinK& g, const CoefK& C, const StateK& S,
                                         int i, int j)
{
    if (i < 0 || i >= g.nr || j < 0 || j >= g.nz) return 0.f;
    const size_t c = (size_t)i * g.P + j;
    return g.dt * bvz_at(C, g, i, j) * S.vz[c];
}

// on d trr/dr at v_r (i,j): odd extension about the axis
__device__ __forceinline__ float adj_x0(const WinK& g, const CoefK& C, const StateK& S,
                                        int i, int j)
{
    float s = 1.f;
    if (i < 0) { i = -i; s = -1.f; }
    if (i == 0 || i >= g.nr) return 0.f;
    float w = adj_w_r(g, C, S, i, j);
    float a = C.ar_int[i];
    if (a != 0.f) w = w + a * (w + C.br_int[i] * S.psi[0][(size_t)i * g.P + j]);
    return s * w;
}

// on d trz/dz at v_r (i,j), i >= 1
__device__ __forceinline__ float adj_x1(const WinK& g, const CoefK& C, const StateK& S,
                                        int i, int j)
{
    if (j < 0 || j >= g.nz) return 0.f;
    float w = adj_w_r(g, C, S, i, j);
    float a = C.az_int[j];
    if (a != 0.f) w = w + a * (w + C.bz_int[j] * S.psi[1][(size_t)i * g.P + j]);
    return w;
}

// on d trz/dr at v_z (i,j): even extension about the axis
__device__ __forceinline__ float adj_x2(const WinK& g, const CoefK& C, const StateK& S,
                                        int i, int j)
{
    if (i < 0) i = -1 - i;
    if (i >= g.nr) return 0.f;
    float w = adj_w_z(g, C, S, i, j);
    float a = C.ar_half[i];
    if (a != 0.f) w = w + a * (w + C.br_half[i] * S.psi[2][(size_t)i * g.P + j]);
    return w;
}

// on d tzz/dz at v_z (i,j)
__device__ __forceinline__ float adj_x3(const WinK& g, const CoefK& C, const StateK& S,
                                        int i, int j)
{
    if (j < 0 || j >= g.nz) return 0.f;
    float w = adj_w_z(g, C, S, i, j);
    float a = C.az_half[j];
    if (a != 0.f) w = w + a * (w + C.bz_half[j] * S.psi[3][(size_t)i * g.P + j]);
    return w;
}

// Transpose of the velocity step at reverse step n: S.{vr,vz} hold
// dJ/dv^{n+1/2}; S.{trr..trz} accumulate to dJ/dtau^n.  Then the residual
// of step n-1 is injected at the receivers (transpose of the recording).
__global__ void __launch_bounds__(256) k_adj_vel(WinK g, CoefK C, StateK S, AdjK q)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nr || j >= g.nz) return;
    const size_t c = (size_t)i * g.P + j;

    // cell (i,j)
    float hoop = 0.5f * (adj_w_r(g, C, S, i, j) * (i >= 1 ? C.inv_r_int[i] : 0.f) +
                         adj_w_r(g, C, S, i + 1, j) * (i + 1 < g.nr ? C.inv_r_int[i + 1] : 0.f));
    float arr = d4(adj_x0(g, C, S, i, j), adj_x0(g, C, S, i + 1, j), adj_x0(g, C, S, i - 1, j),
                   adj_x0(g, C, S, i + 2, j)) * g.inv_dr;
    float azz = d4(adj_x3(g, C, S, i, j - 1), adj_x3(g, C, S, i, j), adj_x3(g, C, S, i, j - 2),
                   adj_x3(g, C, S, i, j + 1)) * g.inv_dz;
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

    // shear node (i,j)
    if (i >= 1) {
        float s = d4(adj_x1(g, C, S, i, j), adj_x1(g, C, S, i, j + 1), adj_x1(g, C, S, i, j - 1),
                     adj_x1(g, C, S, i, j + 2)) * g.inv_dz;
        s += d4(adj_x2(g, C, S, i - 1, j), adj_x2(g, C, S, i, j), adj_x2(g, C, S, i - 2, j),
                adj_x2(g, C, S, i + 1, j)) * g.inv_dr;
        s += 0.5f * (adj_w_z(g, C, S, i - 1, j) * C.inv_r_half[i - 1] +
                     adj_w_z(g, C, S, i, j) * C.inv_r_half[i]);
        S.trz[c] += s;
    }

    // adjoint memories of the velocity step at the own velocity nodes
    if (i >= 1) {
        float w = adj_w_r(g, C, S, i, j);
        if (C.ar_int[i] != 0.f) S.psi_w[0][c] = w + C.br_int[i] * S.psi[0][c];
        if (C.az_int[j] != 0.f) S.psi_w[1][c] = w + C.bz_int[j] * S.psi[1][c];
    }
    {
        float w = adj_w_z(g, C, S, i, j);
        if (C.ar_half[i] != 0.f) S.psi_w[2][c] = w + C.br_half[i] * S.psi[2][c];
        if (C.az_half[j] != 0.f) S.psi_w[3][c] = w + C.bz_half[j] * S.psi[3][c];
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
