// Small kernels of libbh: model setup (Eq. 3, Eq. 4 and the material
// averages), misfit (Eq. 1, Eq. 5), diagonal preconditioner, and the
// gradient-descent update (Eq. 9-12).  Reductions run in one block with a
// fixed traversal order so that their results do not depend on scheduling.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bh {

constexpr int kRedThreads = 1024;

// lambda, mu (Eq. 3, Eq. 4) per cell from velocities and density
__device__ __forceinline__ void lame_f32(float vp, float vs, float rho, float* lam, float* mu)
{
    *mu = rho * vs * vs;
    *lam = rho * vp * vp - 2.f * rho * vs * vs;
}

// lambda, mu and rho per cell; the caller's Vp, Vs are kept as given (cells
// that no update touches report them back unchanged)
__global__ void k_setup_cells(int n, const float* __restrict__ vp, const float* __restrict__ vs,
                              const float* __restrict__ rho, float* lam, float* mu,
                              float* rho_out, float* vp_out, float* vs_out)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float r = rho[k], a = vp[k], b = vs[k];
    rho_out[k] = r;
    vp_out[k] = a;
    vs_out[k] = b;
    lame_f32(a, b, r, &lam[k], &mu[k]);
}

// buoyancy at v_r / v_z nodes and harmonic mu at trz nodes of the global
// model; at the global axial edge the last node row sees its own cells only
__global__ void k_setup_nodes(int nr, int nzg, const float* __restrict__ mu,
                              const float* __restrict__ rho, float* bvr, float* bvz, float* muh)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nr || j >= nzg) return;
    size_t c = (size_t)i * nzg + j;
    int jp = (j + 1 < nzg) ? j + 1 : nzg - 1;
    size_t cp = (size_t)i * nzg + jp;
    bvz[c] = 0.5f * (1.f / rho[c] + 1.f / rho[cp]);
    if (i >= 1) {
        bvr[c] = 0.5f * (1.f / rho[c - nzg] + 1.f / rho[c]);
        float q0 = mu[c - nzg], q1 = mu[c], q2 = mu[cp - nzg], q3 = mu[cp];
        if (q0 <= 0.f || q1 <= 0.f || q2 <= 0.f || q3 <= 0.f) muh[c] = 0.f;
        else muh[c] = 4.f / (1.f / q0 + 1.f / q1 + 1.f / q2 + 1.f / q3);
    } else {
        bvr[c] = 0.f;
        muh[c] = 0.f;
    }
}

// Shifted copies of the node and cell coefficients, [4][5][nr][Pw]:
// lambda, mu, harmonic mu at trz nodes, buoyancy at v_r and v_z nodes of the
// global model; copy k holds global column c - k at column c (zero outside
// the model), so a window starting at global column z0 reads copy
// (4 - z0 % 4) % 4 from a 16-byte aligned column.  blockIdx.z = copy.
__global__ void k_shift_coefs(int nr, int nzg, int Pw, const float* __restrict__ lam,
                              const float* __restrict__ mu, const float* __restrict__ muh,
                              const float* __restrict__ bvr, const float* __restrict__ bvz,
                              float* out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nr || c >= Pw) return;
    const int k = blockIdx.z;
    const size_t pl = (size_t)nr * Pw;
    float* o = out + (size_t)k * 5 * pl + (size_t)i * Pw + c;
    const int j = c - k;
    const bool in = j >= 0 && j < nzg;
    const size_t cg = (size_t)i * nzg + j;
    o[0] = in ? lam[cg] : 0.f;
    o[pl] = in ? mu[cg] : 0.f;
    o[2 * pl] = in ? muh[cg] : 0.f;
    o[3 * pl] = in ? bvr[cg] : 0.f;
    o[4 * pl] = in ? bvz[cg] : 0.f;
}

// inversion mask: formation cell (vs > 0), outside the radial C-PML, and
// inside the axial interior of at least one shot window (colcov[j] != 0)
__global__ void k_setup_mask(int nr, int nzg, int npml_r, const float* __restrict__ vs,
                             const uint8_t* __restrict__ colcov, uint8_t* mask)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nr || j >= nzg) return;
    size_t c = (size_t)i * nzg + j;
    mask[c] = (vs[c] > 0.f && i < nr - npml_r && colcov[j]) ? 1 : 0;
}

__device__ __forceinline__ void block_reduce_max(double* sh, double v)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
}

// max over all entries of a float array (for the CFL check and C-PML d0)
__global__ void __launch_bounds__(kRedThreads) k_max_f32(size_t n, const float* __restrict__ a,
                                                         double* out)
{
    __shared__ double sh[kRedThreads];
    double m = -1e300;
    for (size_t k = threadIdx.x; k < n; k += blockDim.x) m = fmax(m, (double)a[k]);
    block_reduce_max(sh, m);
    if (threadIdx.x == 0) *out = sh[0];
}

// Eq. 5 residual and Eq. 1 misfit, J summed in FP64 in a fixed order:
// thread t adds elements t, t + T, t + 2T, ... then a fixed binary tree.
// resid may alias mod (each element is read, then written, by one thread).
__global__ void __launch_bounds__(kRedThreads) k_misfit(size_t n, const float* mod,
                                                        const float* __restrict__ obs,
                                                        float* resid, double* J)
{
    __shared__ double sh[kRedThreads];
    double s = 0.0;
    for (size_t k = threadIdx.x; k < n; k += blockDim.x) {
        float d = mod[k] - obs[k];
        resid[k] = d;
        s += (double)d * (double)d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *J = 0.5 * sh[0];
}

// Masked maxima over many blocks: each block writes its maxima to
// part[q * gridDim.x + blockIdx.x]; a one-block pass takes the maximum of the
// parts.  A maximum is exact in any order, so the result does not depend on
// the grid.
constexpr int kPartThreads = 256;
constexpr int kMaxParts = 608;  // blocks of the first pass at most

template <int NQ>
__device__ __forceinline__ void block_max_parts(double (&v)[NQ], double* part)
{
    __shared__ double sh[kPartThreads];
    for (int q = 0; q < NQ; ++q) {
        block_reduce_max(sh, v[q]);
        if (threadIdx.x == 0) part[q * gridDim.x + blockIdx.x] = sh[0];
        __syncthreads();
    }
}

template <int NQ>
__device__ __forceinline__ void finish_max_parts(const double* part, int nparts, double (&r)[NQ])
{
    __shared__ double sh[kPartThreads];
    for (int q = 0; q < NQ; ++q) {
        double m = 0.0;
        for (int k = threadIdx.x; k < nparts; k += blockDim.x) m = fmax(m, part[q * nparts + k]);
        block_reduce_max(sh, m);
        r[q] = sh[0];
        __syncthreads();
    }
}

// pass 1 of the masked maxima max |H_lam|, max |H_mu|
__global__ void __launch_bounds__(kPartThreads) k_masked_max2_part(size_t n, const uint8_t* __restrict__ mask,
                                                                   const double* __restrict__ a,
                                                                   const double* __restrict__ b,
                                                                   double* part)
{
    double v[2] = {0.0, 0.0};
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        if (mask[k]) {
            v[0] = fmax(v[0], fabs(a[k]));
            v[1] = fmax(v[1], fabs(b[k]));
        }
    block_max_parts<2>(v, part);
}

// pass 2: out[0] = max H_lam, out[1] = max H_mu
__global__ void __launch_bounds__(kPartThreads) k_masked_max2_finish(const double* __restrict__ part,
                                                                     int nparts, double* out)
{
    double r[2];
    finish_max_parts<2>(part, nparts, r);
    if (threadIdx.x == 0) {
        out[0] = r[0];
        out[1] = r[1];
    }
}

// g <- g / (H + eps max H) inside the mask, 0 outside
__global__ void k_precondition(size_t n, const uint8_t* __restrict__ mask,
                               const double* __restrict__ H_lam, const double* __restrict__ H_mu,
                               const double* __restrict__ hmax, double eps, double* g_lam,
                               double* g_mu)
{
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (!mask[k]) {
        g_lam[k] = 0.0;
        g_mu[k] = 0.0;
        return;
    }
    double dl = H_lam[k] + eps * hmax[0];
    double dm = H_mu[k] + eps * hmax[1];
    g_lam[k] = dl > 0.0 ? g_lam[k] / dl : 0.0;
    g_mu[k] = dm > 0.0 ? g_mu[k] / dm : 0.0;
}

// step lengths alpha_m = kappa max|m| / max|g_m| over the mask: pass 1
__global__ void __launch_bounds__(kPartThreads) k_update_alpha_part(size_t n, const uint8_t* __restrict__ mask,
                                                                    const float* __restrict__ lam,
                                                                    const float* __restrict__ mu,
                                                                    const double* __restrict__ g_lam,
                                                                    const double* __restrict__ g_mu,
                                                                    double* part)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        if (mask[k]) {
            v[0] = fmax(v[0], fabs((double)lam[k]));
            v[1] = fmax(v[1], fabs((double)mu[k]));
            v[2] = fmax(v[2], fabs(g_lam[k]));
            v[3] = fmax(v[3], fabs(g_mu[k]));
        }
    block_max_parts<4>(v, part);
}

// pass 2: alpha[0], alpha[1]
__global__ void __launch_bounds__(kPartThreads) k_update_alpha_finish(const double* __restrict__ part,
                                                                      int nparts, double kappa,
                                                                      double* alpha)
{
    double r[4];
    finish_max_parts<4>(part, nparts, r);
    if (threadIdx.x == 0) {
        alpha[0] = r[2] > 0.0 ? kappa * r[0] / r[2] : 0.0;
        alpha[1] = r[3] > 0.0 ? kappa * r[1] / r[3] : 0.0;
    }
}

// Eq. 9, Eq. 10 inside the mask, then mu >= 0, lambda + 2 mu >= rho (1 m/s)^2,
// and the cell's velocities from Eq. 11, Eq. 12 (cells outside the mask keep
// theirs)
__global__ void k_update_apply(size_t n, const uint8_t* __restrict__ mask,
                               const double* __restrict__ g_lam, const double* __restrict__ g_mu,
                               const double* __restrict__ alpha, const float* __restrict__ rho,
                               float* lam, float* mu, float* vp, float* vs)
{
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || !mask[k]) return;
    double l = (double)lam[k] - alpha[0] * g_lam[k];
    double m = (double)mu[k] - alpha[1] * g_mu[k];
    if (m < 0.0) m = 0.0;
    double floor = (double)rho[k] - 2.0 * m;
    if (l < floor) l = floor;
    const float lf = (float)l, mf = (float)m;
    lam[k] = lf;
    mu[k] = mf;
    const double r = rho[k];
    vp[k] = (float)sqrt(((double)lf + 2.0 * (double)mf) / r);
    vs[k] = (float)sqrt((double)mf / r);
}

// Starting model (Numerical Examples, Fig. 3, Fig. 4): per depth j, the
// velocities at the borehole wall and at r_far, linear in r in between (no
// fused multiply-add, so the rounding is that of the plain expression), the
// far values beyond, the fluid in the cells whose centre lies inside the wall.
__global__ void k_starting_model(int nr, int nz, double dr, double r_wall, double r_far,
                                 const float* __restrict__ vp_wall,
                                 const float* __restrict__ vs_wall,
                                 const float* __restrict__ vp_far,
                                 const float* __restrict__ vs_far, float vp_fluid, float* vp,
                                 float* vs)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nr || j >= nz) return;
    const size_t c = (size_t)i * nz + j;
    const double r = __dmul_rn(i + 0.5, dr);
    if (r < r_wall) {
        vp[c] = vp_fluid;
        vs[c] = 0.f;
        return;
    }
    const double t = fmin(fmax(__ddiv_rn(__dsub_rn(r, r_wall), __dsub_rn(r_far, r_wall)), 0.0), 1.0);
    const double pw = vp_wall[j], sw = vs_wall[j];
    vp[c] = (float)__dadd_rn(pw, __dmul_rn(t, __dsub_rn((double)vp_far[j], pw)));
    vs[c] = (float)__dadd_rn(sw, __dmul_rn(t, __dsub_rn((double)vs_far[j], sw)));
}

// ---- update in (Vp, Vs) and optionally rho (Eq. 9, Eq. 10 applied to the
// velocities; chain rule of Eq. 3, Eq. 4 in FP64)

struct VelGrad {
    double vp, vs, rho;
};

__device__ __forceinline__ VelGrad vel_grad(double vp, double vs, double rho, double gl, double gm,
                                            double gr)
{
    VelGrad g;
    g.vp = 2.0 * rho * vp * gl;
    g.vs = 2.0 * rho * vs * (gm - 2.0 * gl);
    g.rho = gr + (vp * vp - 2.0 * vs * vs) * gl + vs * vs * gm;
    return g;
}

// pass 1: masked maxima of |Vp|, |Vs|, |rho|, |g_Vp|, |g_Vs|, |g_rho|
__global__ void __launch_bounds__(kPartThreads) k_vupdate_part(
    size_t n, const uint8_t* __restrict__ mask, const float* __restrict__ vp,
    const float* __restrict__ vs, const float* __restrict__ rho, const double* __restrict__ g_lam,
    const double* __restrict__ g_mu, const double* __restrict__ g_rho, double* part)
{
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        if (mask[k]) {
            const double a = vp[k], b = vs[k], r = rho[k];
            const VelGrad g = vel_grad(a, b, r, g_lam[k], g_mu[k], g_rho ? g_rho[k] : 0.0);
            v[0] = fmax(v[0], fabs(a));
            v[1] = fmax(v[1], fabs(b));
            v[2] = fmax(v[2], fabs(r));
            v[3] = fmax(v[3], fabs(g.vp));
            v[4] = fmax(v[4], fabs(g.vs));
            v[5] = fmax(v[5], fabs(g.rho));
        }
    block_max_parts<6>(v, part);
}

// pass 2: alpha[0..2] for Vp, Vs, rho (alpha[2] = 0 unless rho steps)
__global__ void __launch_bounds__(kPartThreads) k_vupdate_finish(const double* __restrict__ part,
                                                                 int nparts, double kappa,
                                                                 int update_rho, double* alpha)
{
    double r[6];
    finish_max_parts<6>(part, nparts, r);
    if (threadIdx.x == 0) {
        for (int q = 0; q < 3; ++q) alpha[q] = r[3 + q] > 0.0 ? kappa * r[q] / r[3 + q] : 0.0;
        if (!update_rho) alpha[2] = 0.0;
    }
}

// pass 3: the step inside the mask, clamps Vs >= 0, Vp >= 1 m/s,
// rho >= 1 kg/m^3, then lambda, mu by Eq. 3, Eq. 4 (FP32, as at set-up)
__global__ void k_vupdate_apply(size_t n, const uint8_t* __restrict__ mask,
                                const double* __restrict__ g_lam, const double* __restrict__ g_mu,
                                const double* __restrict__ g_rho, const double* __restrict__ alpha,
                                int update_rho, float* vp, float* vs, float* rho, float* lam,
                                float* mu)
{
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || !mask[k]) return;
    const double a = vp[k], b = vs[k], r = rho[k];
    const VelGrad g = vel_grad(a, b, r, g_lam[k], g_mu[k], g_rho ? g_rho[k] : 0.0);
    const float na = (float)fmax(a - alpha[0] * g.vp, 1.0);
    const float nb = (float)fmax(b - alpha[1] * g.vs, 0.0);
    const float nr = update_rho ? (float)fmax(r - alpha[2] * g.rho, 1.0) : rho[k];
    vp[k] = na;
    vs[k] = nb;
    rho[k] = nr;
    lame_f32(na, nb, nr, &lam[k], &mu[k]);
}

}  // namespace bh

// ------------------------------------------------ checkpoint snapshot codec
//
// Checkpoint snapshots can be stored in 16 bits.  Every plane of every shot
// (6 wavefields and 8 C-PML memories) gets its own scale, a power of two so
// that scaling is exact: FP16 stores x / s with s = 2^(e - 14) where
// 2^e >= max|x| (so the stored values stay below 2^14, inside FP16's range
// with headroom); BF16, which has FP32's exponent range, stores x / 2^e.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace bh {

// max |x| of each plane: one block per plane
__global__ void __launch_bounds__(256) k_plane_maxabs(const float* __restrict__ src,
                                                      size_t plane, float* maxabs)
{
    __shared__ float sh[256];
    const float* p = src + (size_t)blockIdx.x * plane;
    float m = 0.f;
    for (size_t k = threadIdx.x; k < plane; k += blockDim.x) m = fmaxf(m, fabsf(p[k]));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) maxabs[blockIdx.x] = sh[0];
}

// power-of-two scale of a plane from its max |x| (prec 1: BF16, 2: FP16),
// kept a normal FP32 number (exponent >= -126) so that 1/s is finite too;
// a plane below 2^-112 then keeps its values to FP16's subnormal range
__device__ __forceinline__ float snap_scale(float maxabs, int prec)
{
    if (!(maxabs > 0.f) || !(maxabs < 3.0e38f)) return 1.f;
    int e;
    frexpf(maxabs, &e);  // maxabs = f * 2^e, 0.5 <= f < 1
    return ldexpf(1.f, max(prec == 2 ? e - 14 : e, -126));
}

__global__ void k_snap_encode(const float* __restrict__ src, size_t plane, size_t n,
                              const float* __restrict__ maxabs, int prec, uint16_t* dst)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        const float inv = 1.f / snap_scale(maxabs[k / plane], prec);  // exact: power of two
        const float x = src[k] * inv;
        uint16_t q;
        if (prec == 2) q = __half_as_ushort(__float2half_rn(x));
        else q = __bfloat16_as_ushort(__float2bfloat16_rn(x));
        dst[k] = q;
    }
}

__global__ void k_snap_decode(const uint16_t* __restrict__ src, size_t plane, size_t n,
                              const float* __restrict__ maxabs, int prec, float* dst)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        const float s = snap_scale(maxabs[k / plane], prec);
        const uint16_t q = src[k];
        const float x = prec == 2 ? __half2float(__ushort_as_half(q))
                                  : __bfloat162float(__ushort_as_bfloat16(q));
        dst[k] = x * s;
    }
}

}  // namespace bh

namespace bh {

// Gradients with respect to (Vp, Vs, rho) from those with respect to
// (lambda, mu, rho), by Eq. 3 and Eq. 4: lambda = rho (Vp^2 - 2 Vs^2),
// mu = rho Vs^2.  g_rho may be null (then rho is held fixed: output 0).
// Vp, Vs are the model's own velocities (as given, or as the last update
// left them).
__global__ void k_velocity_gradient(size_t n, const float* __restrict__ vp,
                                    const float* __restrict__ vs, const float* __restrict__ rho,
                                    const double* __restrict__ g_lam,
                                    const double* __restrict__ g_mu,
                                    const double* __restrict__ g_rho, float* g_vp, float* g_vs,
                                    float* g_rho_v)
{
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const VelGrad g = vel_grad(vp[k], vs[k], rho[k], g_lam[k], g_mu[k], g_rho ? g_rho[k] : 0.0);
    if (g_vp) g_vp[k] = (float)g.vp;
    if (g_vs) g_vs[k] = (float)g.vs;
    if (g_rho_v) g_rho_v[k] = (float)g.rho;
}

}  // namespace bh
