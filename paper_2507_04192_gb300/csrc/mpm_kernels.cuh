// CUDA kernels of the explicit MPM step, templated on the real type R
// (float or double) and the dimension D (2 or 3).  Included once per
// precision by mpm_kernels_f32.cu / mpm_kernels_f64.cu.
//
// Step (Sec. 2.2): P2G scatters mass, APIC momentum (Appendix B) and the
// stress force of Eq. semi into a shared-memory window of the grid per tile of
// sorted particles, then adds the window to the global grid with one vector
// atomic per touched node; the grid update turns node momentum into velocity
// with gravity and the wall contact of Eq. coulomb_friction; G2P gathers the
// node velocities back to the particles and applies the velocity gradient of
// Eq. update_v_gradient to position, deformation gradient, density and stress.
#pragma once

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "mpm_internal.cuh"

// Resident P2G blocks per SM the 3D single-precision kernel is compiled for.
#ifndef MPM_P2G_MINB
#define MPM_P2G_MINB 3
#endif
// Resident G2P blocks per SM the single-precision kernel is compiled for.
#ifndef MPM_G2P_MINB
#define MPM_G2P_MINB 2
#endif

namespace mpm {

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ float rfloor(float v) { return floorf(v); }
__device__ __forceinline__ double rfloor(double v) { return floor(v); }
__device__ __forceinline__ float rsqrt_(float v) { return sqrtf(v); }
__device__ __forceinline__ double rsqrt_(double v) { return sqrt(v); }
__device__ __forceinline__ bool rfinite(float v) { return isfinite(v); }
__device__ __forceinline__ bool rfinite(double v) { return isfinite(v); }

__device__ __forceinline__ void red_add4(R4<float> *addr, float a, float b, float c, float d)
{
    atomicAdd(reinterpret_cast<float4 *>(addr), make_float4(a, b, c, d));
}
__device__ __forceinline__ void red_add4(R4<double> *addr, double a, double b, double c, double d)
{
    atomicAdd(&addr->x, a);
    atomicAdd(&addr->y, b);
    atomicAdd(&addr->z, c);
    atomicAdd(&addr->w, d);
}

// First stencil cell b = floor(x / dx - 0.5), clamped to [-1, N - 1] (a NaN or
// infinite position therefore still yields an in-grid index).
template <class R>
__device__ __forceinline__ int base_cell(R x, R inv_dx, int N)
{
    int b = (int)rfloor(x * inv_dx - R(0.5));
    return min(max(b, -1), N - 1);
}

// Quadratic B-spline weights of the three stencil nodes at offset fx = x/dx - b
// and their derivatives with respect to x (closed form of the spline of Sec. 2.1
// on [0.5, 1.5)).
template <class R>
__device__ __forceinline__ void bspline(R fx, R inv_dx, R w[3], R dw[3])
{
    const R a = R(1.5) - fx, b = fx - R(1), c = fx - R(0.5);
    w[0] = R(0.5) * a * a;
    w[1] = R(0.75) - b * b;
    w[2] = R(0.5) * c * c;
    dw[0] = -a * inv_dx;
    dw[1] = R(-2) * b * inv_dx;
    dw[2] = c * inv_dx;
}

// Tait pressure p = (K / gamma) ((rho / rho0)^gamma - 1).
template <class R>
__device__ __forceinline__ R tait(const Params<R> &P, R rho)
{
    const R r = rho * P.inv_rho0;
    R rg;
    if (P.gamma_int > 0) {                       // r^gamma by repeated squaring (gamma = 7: three rounds)
        rg = R(1);
        R base = r;
        for (int e = P.gamma_int; e != 0; e >>= 1) {
            if (e & 1) rg *= base;
            base *= base;
        }
    } else {
        rg = pow(r, P.gamma);
    }
    return P.K_over_gamma * (rg - R(1));
}

template <int D> __device__ __forceinline__ int64_t lin3(const int a[3], const int G[3])
{
    if constexpr (D == 2) return (int64_t)a[1] * G[0] + a[0];
    return ((int64_t)a[2] * G[1] + a[1]) * G[0] + a[0];
}

// Friction coefficient of the wall segment holding node a (a-space).
template <class R, int D>
__device__ __forceinline__ R wall_mu(const Params<R> &P, int w, int sim, const int a[3])
{
    const WallDev &wd = P.wall[w];
    if (wd.mu == nullptr) return R(0);
    int s[2] = {0, 0};
#pragma unroll
    for (int q = 0; q < D - 1; ++q) {
        const int ax = wd.seg_axis[q];
        const int c = a[ax] - 2;                       // node coordinate / dx
        int sq = c > 0 ? (int)(((int64_t)c * wd.n_seg[q]) / P.n_cells[ax]) : 0;
        s[q] = min(sq, wd.n_seg[q] - 1);
    }
    const int64_t per_sim = (int64_t)wd.n_seg[0] * wd.n_seg[1];
    return static_cast<const R *>(wd.mu)[sim * per_sim + (int64_t)s[1] * wd.n_seg[0] + s[0]];
}

// Component offsets of the particle state, the order the host sets up: what G2P
// reads first (x, F, rho, and sigma, eps for Drucker-Prager), then v and C.
template <int D, int MAT> struct Lay {
    static constexpr int X = 0, F = D, RHO = D + D * D, SIG = RHO + 1, EPS = RHO + 7;
    static constexpr int V = MAT == 1 ? RHO + 8 : RHO + 1, C = V + D, NC = C + D * D;
    static constexpr int G2P_IN = V;             // G2P reads components [0, G2P_IN)
};

// ------------------------------------------------------------------ TMA / mbarrier helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(phase)
                 : "memory");
    return ok != 0u;
}
// One poll that may suspend the thread for at most about kPollNs nanoseconds
// while the phase is incomplete (the suspend-time hint of mbarrier.try_wait).
constexpr int kPollNs = 1000;
__device__ __forceinline__ bool mbar_poll(uint64_t *bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(phase), "n"(kPollNs)
                 : "memory");
    return ok != 0u;
}
// Bounded wait: false after kMaxWaitIters unsuccessful polls of at most about
// kPollNs each, i.e. about one second.  A copy that completes normally takes
// microseconds.
constexpr int kMaxWaitIters = 1 << 20;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase)
{
    for (int it = 0; it < kMaxWaitIters; ++it)
        if (mbar_poll(bar, phase)) return true;
    return false;
}

// Adds the block-wide sums of v[0..K) to out[slot[k]] (double atomics from one
// thread).  Every thread of the block must call it.
template <int K>
__device__ __forceinline__ void block_sum_add(double (&v)[K], double *out, const int (&slot)[K])
{
    __shared__ double red[32][K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[wid][k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = lane < nw ? red[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0 && t != 0.0) atomicAdd(out + slot[k], t);
        }
    }
}
// TMA tiled load of the grid window of one tile: coordinates (component, node x, y, [z], sim).
__device__ __forceinline__ void tma_load_window(void *dst, const CUtensorMap *map, const int org[3], int sim,
                                                int dim, uint64_t *bar)
{
    if (dim == 3) {
        asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
                     "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(org[0]), "r"(org[1]), "r"(org[2]), "r"(sim),
                     "r"(smem_u32(bar))
                     : "memory");
    } else {
        asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
                     "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(org[0]), "r"(org[1]), "r"(sim),
                     "r"(smem_u32(bar))
                     : "memory");
    }
}

// One-dimensional bulk copy global -> shared (16-byte aligned addresses, size a
// multiple of 16), completion counted on an mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Stage the first ng components of the particle blocks covering slots
// [a, a + count) (a a multiple of kPB) into a shared buffer, block after block
// (ng kPB reals each: particle a + l's component c at buf[(l / kPB) ng kPB + c kPB
// + l % kPB]).  Issued by warp 0: lane 0 sets the expected bytes, lane k copies
// block k with one bulk copy.
template <class R>
__device__ __forceinline__ void stage_blocks(R *buf, const R *__restrict__ S, int ncomp, int ng, int64_t a, int count,
                                             uint64_t *bar)
{
    const int nblk = (count + kPB - 1) / kPB;
    const uint32_t bytes = (uint32_t)(ng * kPB * sizeof(R));
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            mbar_expect_tx(bar, (uint32_t)nblk * bytes);
        }
        __syncwarp();
        for (int k = threadIdx.x; k < nblk; k += 32)
            bulk_g2s(buf + (int64_t)k * ng * kPB, S + ((a >> 5) + k) * (int64_t)ncomp * kPB, bytes, bar);
    }
}

// ------------------------------------------------------------------ P2G

// Separable form of one particle's P2G contribution.  With per-axis weights
// w_a[j] and derivatives dw_a[j] (j = stencil offset), node k receives
//   mass      m_p w_0[k0] w_1[k1] (w_2[k2])
//   momentum  sum_b E[a][b][k_b] prod_{c != b} w_c[k_c]       (component a)
// where E[a][b][j] = m_p C_ab dx j w_b[j] + Fm_ab dw_b[j] (+ m_p u0_a w_b[j] for b = 0),
// u0 = v_p - C_p fx dx and Fm = -dt V_p sigma_p.  This is m_p w (v_p + C_p (x_i - x_p))
// - dt V_p sigma_p grad w expanded over the tensor-product weights.
template <class R, int D> struct P2GFactors {
    int b[D];
    R w[D][3];
    R E[D][D][3];
};

// Components of the particle state P2G reads, in staging order: x (D), v (D),
// C (D^2), rho, and for Drucker-Prager sigma (6).  x, v, C are consecutive in
// the state, as are rho and sigma.
template <int D> __host__ __device__ __forceinline__ constexpr int p2g_ncomp(int material)
{
    return 2 * D + D * D + 1 + (material == 1 ? 6 : 0);
}
// State component of P2G staging slot j (x, v, C, rho, sigma).
template <int D, int MAT> __host__ __device__ __forceinline__ constexpr int p2g_comp(int j)
{
    using Ly = Lay<D, MAT>;
    return j < D ? Ly::X + j
                 : (j < 2 * D ? Ly::V + (j - D)
                              : (j < 2 * D + D * D ? Ly::C + (j - 2 * D)
                                                   : (j == 2 * D + D * D ? Ly::RHO : Ly::SIG + (j - 2 * D - D * D - 1))));
}

// P2G factors of one particle from its raw components raw(j) (staging order).
// MAT = 0 (fluid) or 1 (Drucker-Prager) fixes the material at compile time; -1 reads it from P.
template <class R, int D, int MAT = -1, class Raw>
__device__ __forceinline__ void p2g_factors(const Params<R> &P, Raw raw, P2GFactors<R, D> &f)
{
    constexpr int J_RHO = 2 * D + D * D;
    R x[D], v[D], C[D * D], Fm[D * D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        x[a] = raw(a);
        v[a] = raw(D + a);
    }
#pragma unroll
    for (int q = 0; q < D * D; ++q) C[q] = raw(2 * D + q);
    const R rho = raw(J_RHO);
    const R Vp = P.mass / rho;
    if (MAT >= 0 ? MAT == 0 : P.material == 0) {
        const R c = P.dt * Vp * tait(P, rho);          // -dt V (-p I)
#pragma unroll
        for (int q = 0; q < D * D; ++q) Fm[q] = (q % (D + 1) == 0) ? c : R(0);
    } else {
        R s6[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) s6[k] = raw(J_RHO + 1 + k);
        const R c = -P.dt * Vp;
        if constexpr (D == 2) {
            Fm[0] = c * s6[0]; Fm[1] = c * s6[3];
            Fm[2] = c * s6[3]; Fm[3] = c * s6[1];
        } else {
            Fm[0] = c * s6[0]; Fm[1] = c * s6[3]; Fm[2] = c * s6[4];
            Fm[3] = c * s6[3]; Fm[4] = c * s6[1]; Fm[5] = c * s6[5];
            Fm[6] = c * s6[4]; Fm[7] = c * s6[5]; Fm[8] = c * s6[2];
        }
    }
    if (P.no_force) {                                   // FLIP's second pass: momentum only
#pragma unroll
        for (int q = 0; q < D * D; ++q) Fm[q] = R(0);
    }
    R fx[D], dw[D][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        f.b[a] = base_cell(x[a], P.inv_dx, P.n_cells[a]);
        fx[a] = x[a] * P.inv_dx - R(f.b[a]);
        bspline(fx[a], P.inv_dx, f.w[a], dw[a]);
    }
    // two forms of the same sums: with hoisted products and chained fused
    // multiply-adds (3D sand P2G 0.1252 -> 0.1231 ms on the 2.76M-particle collapse,
    // 2D 0.170 -> 0.168 ms on the batched dam breaks), or as written below it, which
    // the 3D fluid kernel keeps (the hoisted form raised its spills: 0.098 -> 0.105
    // ms on the 1.92M-particle dam break)
    if constexpr (!(D == 3 && MAT == 0)) {
    const R mp = P.mass, mdx = P.mass * P.dx;
    R fxdx[D];
#pragma unroll
    for (int c2 = 0; c2 < D; ++c2) fxdx[c2] = fx[c2] * P.dx;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        R u0 = v[a];
#pragma unroll
        for (int c2 = 0; c2 < D; ++c2) u0 = fma(-C[a * D + c2], fxdx[c2], u0);
        const R mu0 = mp * u0;
#pragma unroll
        for (int b2 = 0; b2 < D; ++b2) {
            const R mc = C[a * D + b2] * mdx;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                R e = Fm[a * D + b2] * dw[b2][j];
                if (j > 0) e = fma(j == 1 ? mc : mc + mc, f.w[b2][j], e);
                if (b2 == 0) e = fma(mu0, f.w[0][j], e);
                f.E[a][b2][j] = e;
            }
        }
    }
    } else {
    const R mp = P.mass;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        R u0 = v[a];
#pragma unroll
        for (int c2 = 0; c2 < D; ++c2) u0 -= C[a * D + c2] * fx[c2] * P.dx;
#pragma unroll
        for (int b2 = 0; b2 < D; ++b2) {
            const R mc = mp * C[a * D + b2] * P.dx;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                R e = mc * R(j) * f.w[b2][j] + Fm[a * D + b2] * dw[b2][j];
                if (b2 == 0) e += mp * u0 * f.w[0][j];
                f.E[a][b2][j] = e;
            }
        }
    }
    }
}

// Mass and momentum (+ dt force) of stencil node k = (k0, k1, k2).
template <class R, int D>
__device__ __forceinline__ void p2g_node(const P2GFactors<R, D> &f, R mp, int k0, int k1, int k2, R &m, R mom[D])
{
    if constexpr (D == 2) {
        m = mp * f.w[0][k0] * f.w[1][k1];
#pragma unroll
        for (int a = 0; a < D; ++a) mom[a] = f.E[a][0][k0] * f.w[1][k1] + f.w[0][k0] * f.E[a][1][k1];
    } else {
        const R wxy = f.w[0][k0] * f.w[1][k1];
        const R wz = f.w[2][k2];
        m = mp * wxy * wz;
#pragma unroll
        for (int a = 0; a < D; ++a)
            mom[a] = wz * (f.E[a][0][k0] * f.w[1][k1] + f.w[0][k0] * f.E[a][1][k1]) + wxy * f.E[a][2][k2];
    }
}

// Sum one particle's contributions into per-cell register accumulators (its
// base is the cell's base).  Products shared by the three nodes of a z-column
// are formed once per (k0, k1).
template <class R, int D>
__device__ __forceinline__ void p2g_accumulate(const P2GFactors<R, D> &f, R mp, R (&acc)[Geo<D>::STENCIL][D + 1])
{
    if constexpr (D == 2) {
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1)
#pragma unroll
            for (int k0 = 0; k0 < 3; ++k0) {
                const int k = k1 * 3 + k0;
                acc[k][0] = fma(mp * f.w[0][k0], f.w[1][k1], acc[k][0]);
#pragma unroll
                for (int a = 0; a < D; ++a)           // two chained fused multiply-adds per value
                    acc[k][1 + a] = fma(f.E[a][0][k0], f.w[1][k1], fma(f.w[0][k0], f.E[a][1][k1], acc[k][1 + a]));
            }
    } else {
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1)
#pragma unroll
            for (int k0 = 0; k0 < 3; ++k0) {
                const R wxy = f.w[0][k0] * f.w[1][k1];
                const R mwxy = mp * wxy;
                R Tm[D];
#pragma unroll
                for (int a = 0; a < D; ++a) Tm[a] = fma(f.E[a][0][k0], f.w[1][k1], f.w[0][k0] * f.E[a][1][k1]);
#pragma unroll
                for (int k2 = 0; k2 < 3; ++k2) {
                    const int k = (k2 * 3 + k1) * 3 + k0;
                    acc[k][0] = fma(mwxy, f.w[2][k2], acc[k][0]);
#pragma unroll
                    for (int a = 0; a < D; ++a)
                        acc[k][1 + a] = fma(f.w[2][k2], Tm[a], fma(wxy, f.E[a][2][k2], acc[k][1 + a]));
                }
            }
    }
}

// Byte offset of the P2G per-thread staging slots in dynamic shared memory
// (after the window and the cell offsets, 16-byte aligned) and the total size.
template <class R, int D> __host__ __device__ constexpr size_t p2g_stage_offset()
{
    return ((size_t)(D + 1) * Geo<D>::WN * sizeof(R) + (Geo<D>::TN + 1) * sizeof(int32_t) + 15) & ~size_t(15);
}
// Particles in flight per P2G thread (cp.async stages of its staging slots; 3
// measured slower than 2 on the 3D collapse).
#ifndef MPM_P2G_STAGES
#define MPM_P2G_STAGES 2
#endif

template <class R, int D, int NT> __host__ __device__ constexpr size_t p2g_smem_bytes()
{
    return p2g_stage_offset<R, D>() + (size_t)MPM_P2G_STAGES * p2g_ncomp<D>(1) * NT * sizeof(R);
}

template <int D> __device__ __forceinline__ int win_index(const int l[D], int k0, int k1, int k2)
{
    using Gm = Geo<D>;
    if constexpr (D == 2) return (l[1] + k1) * Gm::W + (l[0] + k0);
    else return ((l[2] + k2) * Gm::W + (l[1] + k1)) * Gm::W + (l[0] + k0);
}

// Marks node tile g touched and, the first time, appends it to the list the grid
// update walks.
__device__ __forceinline__ void mark_node_tile(uint32_t *flags, int32_t *list, int32_t *count, int64_t g)
{
    if (flags[g] == 0u && atomicExch(&flags[g], 1u) == 0u) list[atomicAdd(count, 1)] = (int32_t)g;
}

// Scatter one particle's 3^D contributions: shared-memory atomics when its stencil
// lies in the window (l = window coordinates of its base), else global atomics.
template <class R, int D>
__device__ __forceinline__ void p2g_scatter(const Params<R> &P, const P2GFactors<R, D> &f, const int org[3], R *sm,
                                            R4<R> *Asim, uint32_t *flags_sim, bool &escaped)
{
    using Gm = Geo<D>;
    int l[D];
    bool inside = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        l[a] = f.b[a] + 2 - org[a];
        inside = inside && l[a] >= 0 && l[a] <= Gm::W - 3;
    }
    escaped = !inside;
#pragma unroll
    for (int k = 0; k < Gm::STENCIL; ++k) {
        const int k0 = k % 3, k1 = (k / 3) % 3, k2 = k / 9;
        R m, mom[D];
        p2g_node<R, D>(f, P.mass, k0, k1, k2, m, mom);
        if (inside) {
            const int li = win_index<D>(l, k0, k1, k2);
            atomicAdd(&sm[li], m);
#pragma unroll
            for (int a = 0; a < D; ++a) atomicAdd(&sm[(a + 1) * Gm::WN + li], mom[a]);
        } else {
            int a3[3] = {0, 0, 0}, u[3] = {0, 0, 0};
            const int kk[3] = {k0, k1, k2};
#pragma unroll
            for (int a = 0; a < D; ++a) {
                a3[a] = f.b[a] + 2 + kk[a];
                u[a] = a3[a] / Gm::T;
            }
            red_add4(&Asim[lin3<D>(a3, P.G_nodes)], m, mom[0], mom[1], D == 3 ? mom[D - 1] : R(0));
            mark_node_tile(P.flags, P.node_list, P.list_count, (flags_sim - P.flags) + lin3<D>(u, P.node_tiles));
        }
    }
}

// Claim the next tile of the compact list (block-uniform); -1 when done.
__device__ __forceinline__ int next_tile(int32_t *cursor, int n_tiles, int *s_slot)
{
    __syncthreads();
    if (threadIdx.x == 0) *s_slot = atomicAdd(cursor, 1);
    __syncthreads();
    const int k = *s_slot;
    return k < n_tiles ? k : -1;
}

// Per-thread asynchronous copy of one element global -> shared (cp.async), in
// commit groups the issuing thread waits for.
template <class R> __device__ __forceinline__ void cp_async_elem(R *dst, const R *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"((int)sizeof(R))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Walks one thread's particles of a tile: cells c = threadIdx.x, +NT, ... and
// the slots q of each cell (cell_off ranges); next() moves to the next particle.
// (Rotating the cell of each round across the tile's columns, which balances
// tiles cut by the body's edge, measured slower: the warps' cells then straddle
// two layer groups.)
template <int TN, int NT> struct CellCursor {
    int c, q, q1;
    __device__ __forceinline__ void start() { c = (int)threadIdx.x - NT; q = 0; q1 = 0; }
    __device__ __forceinline__ bool next(const int32_t *off)
    {
        ++q;
        while (q >= q1) {
            c += NT;
            if (c >= TN) return false;
            q = off[c];
            q1 = off[c + 1];
        }
        return true;
    }
};

template <int D> constexpr int kP2GStageComps = p2g_ncomp<D>(1);

// P2G.  Blocks of NT threads claim tiles dynamically; one thread per cell.  A
// thread walks its cells' particles (slots from the position map; within a
// group the rank planes are contiguous and cell-ordered, so the copies of a warp
// are coalesced) through a two-stage pipeline: the components of the particle
// after next are copied into the thread's shared-memory slots (cp.async) while
// the current one is summed.  It sums the contributions of the particles still
// in their cell in registers (3^D nodes x (1 + D) values) and adds them to the
// shared-memory window when it leaves the cell.  A particle that has left its
// cell since the sort is scattered on its own: into the window, or straight to
// the grid if it has also left the window.  The window is added to the grid with
// one vector atomic per touched node.  Without REG (FP64 in 3D) every particle
// is scattered on its own.
template <class R, int D, bool REG, int NT, int MAT>
__global__ void __launch_bounds__(NT, (D == 3 && REG) ? MPM_P2G_MINB : 1)
    k_p2g(const Params<R> P, const R *__restrict__ S, const int4 *__restrict__ tiles, int32_t *__restrict__ counters,
          const int32_t *__restrict__ posmap, const int32_t *__restrict__ cell_off, R4<R> *__restrict__ A,
          uint32_t *__restrict__ flags, unsigned long long *__restrict__ escaped_count)
{
    using Gm = Geo<D>;
    constexpr int NCM = kP2GStageComps<D>;
    constexpr int NC = p2g_ncomp<D>(MAT);             // components this material stages
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sm = reinterpret_cast<R *>(smem_raw);
    int32_t *off = reinterpret_cast<int32_t *>(sm + (D + 1) * Gm::WN);
    R *stg = reinterpret_cast<R *>(smem_raw + p2g_stage_offset<R, D>());
    __shared__ uint32_t tile_mask;
    __shared__ int s_slot;
    const int n_tiles = counters[1];
    const int tid = threadIdx.x;
    for (;;) {
        const int k = next_tile(&counters[2], n_tiles, &s_slot);
        if (k < 0) break;
        const int4 t = tiles[k];
        for (int i = tid; i < (D + 1) * Gm::WN; i += NT) sm[i] = R(0);
        for (int c = tid; c <= Gm::TN; c += NT) off[c] = cell_off[(int64_t)k * (Gm::TN + 1) + c];
        if (tid == 0) tile_mask = 0u;
        __syncthreads();
        const int sim = (int)(t.x / P.tiles_per_sim);
        int64_t tl = t.x - (int64_t)sim * P.tiles_per_sim;
        int org[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            org[a] = (int)(tl % P.n_tiles[a]) * Gm::T;
            tl /= P.n_tiles[a];
        }
        R4<R> *Asim = A + (int64_t)sim * P.nodes_per_sim;
        uint32_t *fsim = flags + (int64_t)sim * P.node_tiles_per_sim;
        const int32_t *pmap = posmap + t.y;
        bool any_escape = false;

        R *const Sv = P.save_S == nullptr ? nullptr : P.save_S + t.y;
        auto issue = [&](int stage, int32_t pos) {
            R *dst = stg + stage * NCM * NT + tid;
            const R *src = S + sblock((int64_t)t.y + pos, Lay<D, MAT>::NC);
#pragma unroll
            for (int j = 0; j < NC; ++j) cp_async_elem(dst + j * NT, src + p2g_comp<D, MAT>(j) * kPB);
        };
        // producer: MPM_P2G_STAGES particles ahead of the consumer, its next slot's position prefetched
        CellCursor<Gm::TN, NT> pc, cc;
        pc.start();
        cc.start();
        bool hp = pc.next(off);
#pragma unroll
        for (int s0 = 0; s0 < MPM_P2G_STAGES; ++s0) {
            if (hp) issue(s0, pmap[pc.q]);
            cp_async_commit();
            hp = hp && pc.next(off);
        }
        int32_t ppos = hp ? pmap[pc.q] : 0;

        bool hc = cc.next(off);
        int stage = 0;
        int cur = -1;                                  // cell whose accumulators are live
        int lc[D], bown[D];
        R acc[Gm::STENCIL][D + 1];
        while (hc) {
            if (cc.c != cur) {
                cur = cc.c;
                int r = cur;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const int ci = r % Gm::T;
                    r /= Gm::T;
                    lc[a] = ci + 1;                    // window coordinates of the cell's base
                    bown[a] = org[a] + ci - 1;         // base cell index of the cell
                }
                if constexpr (REG) {
#pragma unroll
                    for (int kk = 0; kk < Gm::STENCIL; ++kk)
#pragma unroll
                        for (int v = 0; v <= D; ++v) acc[kk][v] = R(0);
                }
            }
            cp_async_wait<MPM_P2G_STAGES - 1>();
            P2GFactors<R, D> f;
            {
                const R *src = stg + stage * NCM * NT + tid;
                if (Sv != nullptr) {                   // the adjoint's copy of this step's state
                    R *d = Sv + pmap[cc.q];
#pragma unroll
                    for (int j = 0; j < NC; ++j) d[j * P.n] = src[j * NT];
                }
                p2g_factors<R, D, MAT>(P, [&](int j) { return src[j * NT]; }, f);
            }
            if (hp) issue(stage, ppos);
            cp_async_commit();
            hp = hp && pc.next(off);
            if (hp) ppos = pmap[pc.q];
            bool own = REG;
#pragma unroll
            for (int a = 0; a < D; ++a) own = own && (f.b[a] == bown[a]);
            if (own) {
                if constexpr (REG) p2g_accumulate<R, D>(f, P.mass, acc);
            } else {
                bool esc = false;
                p2g_scatter<R, D>(P, f, org, sm, Asim, fsim, esc);
                any_escape |= esc;
            }
            stage = stage + 1 == MPM_P2G_STAGES ? 0 : stage + 1;
            hc = cc.next(off);
            if constexpr (REG) {
                if (!hc || cc.c != cur) {
#pragma unroll
                    for (int kk = 0; kk < Gm::STENCIL; ++kk) {
                        const int li = win_index<D>(lc, kk % 3, (kk / 3) % 3, kk / 9);
#pragma unroll
                        for (int v = 0; v <= D; ++v) atomicAdd(&sm[v * Gm::WN + li], acc[kk][v]);
                    }
                }
            }
        }
        cp_async_wait<0>();
        const unsigned ball = __ballot_sync(0xffffffffu, any_escape);
        if (ball && (threadIdx.x & 31) == 0) atomicAdd(escaped_count, (unsigned long long)__popc(ball));
        __syncthreads();
        for (int i = threadIdx.x; i < Gm::WN; i += NT) {
            const R m = sm[i];
            const R q0 = sm[Gm::WN + i], q1 = sm[2 * Gm::WN + i];
            const R q2 = D == 3 ? sm[3 * Gm::WN + i] : R(0);
            if (m != R(0) || q0 != R(0) || q1 != R(0) || q2 != R(0)) {
                int l[3] = {0, 0, 0}, a3[3] = {0, 0, 0};
                int r = i;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    l[a] = r % Gm::W;
                    r /= Gm::W;
                    a3[a] = org[a] + l[a];
                }
                red_add4(&Asim[lin3<D>(a3, P.G_nodes)], m, q0, q1, q2);
                unsigned bit = 0;
#pragma unroll
                for (int a = 0; a < D; ++a) bit |= (l[a] >= Gm::T ? 1u : 0u) << a;
                atomicOr(&tile_mask, 1u << bit);
            }
        }
        __syncthreads();
        if (threadIdx.x < (1 << D) && ((tile_mask >> threadIdx.x) & 1u)) {
            int u[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < D; ++a) u[a] = org[a] / Gm::T + ((threadIdx.x >> a) & 1);
            mark_node_tile(flags, P.node_list, P.list_count,
                           (int64_t)sim * P.node_tiles_per_sim + lin3<D>(u, P.node_tiles));
        }
    }
    if (threadIdx.x == 0) counters[3] = 0;         // G2P cursor for the next kernel (G2P follows)
}

// Where k_p2g_direct takes its particles and writes its sums.  Forward P2G (MAT
// = 0 fluid, 1 Drucker-Prager): the state S (stride ld = npad), the current sort
// tables and cursor counters[2], sums into A, node tiles marked.  The adjoint's
// v_bar scatter (MAT = 2): positions from a kept state (stride ld = n) and the
// 21 scatter coefficients per particle from src2 (v_bar_t, C_bar, L_bar), the
// sort tables of that state's generation and its own cursor, sums into the grid
// adjoint, no marks.
template <class R> struct P2GIO {
    const R *S;                       // x (and for P2G the other inputs): component c at S[c ld + slot]
    const R *src2;                    // MAT 2: 21 coefficients, component c at src2[c ld + slot]
    int64_t ld;
    const int4 *tiles;                // compact tiles in key order
    const int32_t *n_tiles;           // their count
    int32_t *cursor;                  // work-item cursor (zero at launch)
    const int32_t *posmap, *cell_off;
    R4<R> *A;                         // sums (per simulation: A + sim * nodes_per_sim)
    uint32_t *flags;                  // node tile flags (MAT 0, 1)
};

// P2G factors of one particle of the adjoint's v_bar scatter (Eq. dzda reversed
// through G2P): the node value v_bar_k = w_k (v_bar_t + (4 / dx) C_bar (k - fx))
// + L_bar grad w_k is P2G's momentum with mass 1, velocity v_bar_t, affine
// matrix (4 / dx^2) C_bar and stress coefficient L_bar.
template <class R, class Raw>
__device__ __forceinline__ void adj_scatter_factors(const Params<R> &P, Raw raw, P2GFactors<R, 3> &f)
{
    constexpr int D = 3;
    R x[D], fx[D], dw[D][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        x[a] = raw(a);
        f.b[a] = base_cell(x[a], P.inv_dx, P.n_cells[a]);
        fx[a] = x[a] * P.inv_dx - R(f.b[a]);
        bspline(fx[a], P.inv_dx, f.w[a], dw[a]);
    }
    const R cs = R(4) * P.inv_dx;                 // C_bar (k - fx) enters as (4 / dx) C_bar (k - fx)
#pragma unroll
    for (int a = 0; a < D; ++a) {
        R u0 = raw(3 + a);
#pragma unroll
        for (int c2 = 0; c2 < D; ++c2) u0 -= cs * raw(6 + a * D + c2) * fx[c2];
#pragma unroll
        for (int b2 = 0; b2 < D; ++b2) {
            const R mc = cs * raw(6 + a * D + b2);
            const R lb = raw(15 + a * D + b2);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                R e = mc * R(j) * f.w[b2][j] + lb * dw[b2][j];
                if (b2 == 0) e += u0 * f.w[0][j];
                f.E[a][b2][j] = e;
            }
        }
    }
}

// A particle that left its sort cell, scattered on its own to the grid (3^D vector
// atomics), with its node tiles marked when flags is set (tbase: the first tile of
// its simulation in the list's numbering over all simulations).  Kept out of line: the
// path is rare and its registers would otherwise count against the accumulating
// loop.  The factors go by value: a reference kept them in local memory for every
// particle (P2G 0.166 -> 0.145 ms on the 2.76M-particle collapse by value; having
// the callee recompute them from the staged slots measured 0.188 ms).
// Node values are stored (m, q) for P2G; with flags == nullptr (the adjoint's v_bar
// scatter, no mass channel) as (q, 0), the grid adjoint's layout.
template <class R, int D>
__device__ __noinline__ void p2g_escape(const P2GFactors<R, D> f, R mass, R4<R> *Asim, int Gx, int Gy,
                                        uint32_t *flags, int64_t tbase, int32_t *list, int32_t *count, int ntx,
                                        int nty)
{
    for (int kk = 0; kk < Geo<D>::STENCIL; ++kk) {
        const int k0 = kk % 3, k1 = (kk / 3) % 3, k2 = D == 3 ? kk / 9 : 0;
        R m, mom[D];
        p2g_node<R, D>(f, mass, k0, k1, k2, m, mom);
        const int a0 = f.b[0] + 2 + k0, a1 = f.b[1] + 2 + k1, a2 = D == 3 ? f.b[D - 1] + 2 + k2 : 0;
        R4<R> *node = &Asim[((int64_t)a2 * Gy + a1) * Gx + a0];
        if (flags != nullptr) red_add4(node, m, mom[0], mom[1], D == 3 ? mom[D - 1] : R(0));
        else red_add4(node, mom[0], mom[1], D == 3 ? mom[D - 1] : R(0), R(0));
        if (D == 3 && flags != nullptr) {        // the list holds tiles by their index over all simulations
            const int u0 = a0 / Geo<D>::T, u1 = a1 / Geo<D>::T, u2 = a2 / Geo<D>::T;
            mark_node_tile(flags, list, count, tbase + ((int64_t)u2 * nty + u1) * ntx + u0);
        }
    }
    // 2D: the node tiles the stencil reaches, each marked once: one or two per
    // axis, nodes b + 2 .. b + 4 (marking the tile of every node waited on 3^D
    // flag loads in turn: P2G 0.1014 -> 0.0988 ms over the first 300 steps of the
    // 256 batched dam breaks, 0.147 -> 0.134 ms over steps 605-905).  3D keeps
    // the tile of every node: with the once-per-tile form the 3D single-precision
    // adjoint runs faulted the GPU (error 717 and an illegal address), for a
    // reason not found by reading; few 3D particles escape, so it gains nothing.
    if (D == 2 && flags != nullptr) {            // the list holds tiles by their index over all simulations
        int lo[3] = {0, 0, 0}, span[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            lo[a] = (f.b[a] + 2) / Geo<D>::T;
            span[a] = (f.b[a] + 4) / Geo<D>::T - lo[a];          // 0 or 1
        }
        for (int mk = 0; mk < (1 << D); ++mk) {
            bool in = true;
#pragma unroll
            for (int a = 0; a < D; ++a) in = in && ((mk >> a) & 1) <= span[a];
            if (!in) continue;
            const int u0 = lo[0] + (mk & 1), u1 = lo[1] + ((mk >> 1) & 1), u2 = lo[2] + ((mk >> 2) & 1);
            mark_node_tile(flags, list, count, tbase + ((int64_t)u2 * nty + u1) * ntx + u0);
        }
    }
}

// Per-cell node sums of k_p2g_direct: 3^D nodes x (m, q).  (Keeping them as float
// pairs added with paired fused multiply-adds, as G2P's contraction does, did not
// pay here: pairs of two velocity components raised the register spills of the
// 168-register 3D kernel, pairs of the nodes k2 = 0, 1 of a column measured the
// same, 0.1251 against 0.1251 ms on the 2.76M-particle collapse.)
template <class R, int D> struct CellSums {
    R acc[Geo<D>::STENCIL][D + 1];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < Geo<D>::STENCIL; ++k)
#pragma unroll
            for (int v = 0; v <= D; ++v) acc[k][v] = R(0);
    }
    __device__ __forceinline__ void add(const P2GFactors<R, D> &f, R mp) { p2g_accumulate<R, D>(f, mp, acc); }
    __device__ __forceinline__ R m(int k) const { return acc[k][0]; }
    __device__ __forceinline__ R q(int k, int a) const { return a < D ? acc[k][1 + a] : R(0); }
};


// Components staged per particle by k_p2g_direct: P2G's inputs (MAT 0, 1), or x
// and the 21 scatter coefficients (MAT 2).
template <int D, int MAT> __host__ __device__ constexpr int direct_stage_comps()
{
    return MAT == 2 ? 24 : kP2GStageComps<D>;
}
// Per warp of k_p2g_direct: its work item's 129 cell offsets (padded to 132),
// staged in shared memory at the start of the item.
constexpr int kDirectOffPad = 132;
// Cells per work item and cp.async stages per thread of the cell-ordered P2G.
// Items of 32 cells give each lane one cell (its cursor walks that cell's
// particles only) and more items to balance the SMs: on the 2.76M-particle
// collapse P2G 0.123 ms with 128-cell items (four cells per lane), 0.118 with 64,
// 0.105 with 32; on the batched 2D dam breaks 0.167 -> 0.152 ms.  In 2D (16
// particles per cell in the dense fluids) the pipeline is one stage deeper.
#ifndef MPM_P2G2_CELLS
#define MPM_P2G2_CELLS 32
#endif
#ifndef MPM_P2G2_STAGES
#define MPM_P2G2_STAGES 3
#endif
#ifndef MPM_P2G3_CELLS
#define MPM_P2G3_CELLS 32
#endif
#ifndef MPM_P2G3_STAGES
#define MPM_P2G3_STAGES 2
#endif
template <int D> __host__ __device__ constexpr int direct_cells() { return D == 3 ? MPM_P2G3_CELLS : MPM_P2G2_CELLS; }
template <int D> __host__ __device__ constexpr int direct_stages() { return D == 3 ? MPM_P2G3_STAGES : MPM_P2G2_STAGES; }
template <class R, int D, int NT, int MAT> __host__ __device__ constexpr size_t p2g_direct_smem()
{
    return (size_t)direct_stages<D>() * direct_stage_comps<D, MAT>() * NT * sizeof(R) +
           (size_t)(NT / 32) * kDirectOffPad * sizeof(int32_t);
}

// P2G without a shared-memory window (register accumulation, single precision).
// Warps claim work items of 128 cells (two layer groups of a 3D tile, half of a
// 2D tile) from a global cursor and never synchronise with each other: lane l
// walks cells base + l, + 32, + 64, + 96 through a two-stage cp.async pipeline,
// sums the particles still in their cell in registers and adds the 3^D node sums
// of a cell straight to the grid with vector atomics (27 per cell in 3D instead
// of 108 shared-memory atomics plus the window pass); particles that left their
// cell are scattered on their own.  The warp marks the node tiles its cells reach.
#ifndef MPM_P2G_DIRECT
#define MPM_P2G_DIRECT 1
#endif
// One work item of the cell-ordered P2G: the CELLS cells [cbase, cbase + CELLS)
// of compact tile k (key order), one warp, lane l walking cells cbase + l + 32 r.
// stg: this block's cp.async staging slots (ST stages x NCM x NT reals); s_off:
// this warp's 132 shared ints for the item's cell offsets.  MAT 2 (the adjoint's
// v_bar scatter) is 3D only.
template <class R, int D, int NT, int MAT>
__device__ __forceinline__ void p2g_direct_item(const Params<R> &P, const P2GIO<R> &io, R *stg, int32_t *s_off,
                                                int k, int cbase, bool &any_escape)
{
    using Gm = Geo<D>;
    constexpr bool ADJ = MAT == 2;
    static_assert(!ADJ || D == 3, "the v_bar scatter is 3D");
    constexpr int NCM = direct_stage_comps<D, MAT>();
    constexpr int NC = ADJ ? 24 : p2g_ncomp<D>(MAT);
    constexpr int CELLS = direct_cells<D>();
    constexpr int ST = direct_stages<D>();
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t ld = io.ld;
    const R mass = ADJ ? R(0) : P.mass;
    const int4 t = io.tiles[k];
    const int sim = (int)(t.x / P.tiles_per_sim);
    int64_t tl = t.x - (int64_t)sim * P.tiles_per_sim;
    int org[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        org[a] = (int)(tl % P.n_tiles[a]) * Gm::T;
        tl /= P.n_tiles[a];
    }
    if constexpr (D == 2) org[2] = 0;
    R4<R> *Asim = io.A + (int64_t)sim * P.nodes_per_sim;
    const int32_t *pmap = io.posmap + t.y;
    const int32_t *goff = io.cell_off + (int64_t)t.w * (Gm::TN + 1) + cbase;   // t.w: index in key order
    // the item's cell offsets, staged once (coalesced) so that the per-cell lookups
    // below are shared-memory reads (staging the position map as well measured
    // slower in 3D, 0.125 -> 0.146 ms on the collapse, and no faster in 2D)
    __syncwarp();
    for (int i = lane; i <= CELLS; i += 32) s_off[i] = goff[i];
    __syncwarp();
    const int32_t *off = s_off - cbase;           // off[c] for the item's cells c in [cbase, cbase + CELLS]
    auto slot = [&](int q) { return pmap[q]; };
    const R *St = io.S + t.y;                     // MAT 2: component-major with stride ld
    const R *S2 = ADJ ? io.src2 + t.y : nullptr;
    R *const Sv = (ADJ || P.save_S == nullptr) ? nullptr : P.save_S + t.y;
    auto issue = [&](int stage, int32_t pos) {
        R *dst = stg + stage * NCM * NT + tid;
        if constexpr (ADJ) {
#pragma unroll
            for (int j = 0; j < 3; ++j) cp_async_elem(dst + j * NT, St + pos + j * ld);
#pragma unroll
            for (int j = 0; j < 21; ++j) cp_async_elem(dst + (3 + j) * NT, S2 + pos + j * ld);
        } else {                                  // the particle state, in blocks of kPB
            const R *src = io.S + sblock((int64_t)t.y + pos, Lay<D, MAT>::NC);
#pragma unroll
            for (int j = 0; j < NC; ++j) cp_async_elem(dst + j * NT, src + p2g_comp<D, MAT>(j) * kPB);
        }
    };
    // cursors over this lane's cells cbase + lane + 32 r and their slots
    struct CurMulti {
        int c, q, q1, end;
        __device__ __forceinline__ bool next(const int32_t *o)
        {
            ++q;
            while (q >= q1) {
                c += 32;
                if (c >= end) return false;
                q = o[c];
                q1 = o[c + 1];
            }
            return true;
        }
    };
    // one cell per lane (32-cell items): the cursor walks that cell's particles only
    struct CurOne {
        int c, q, q1;
        __device__ __forceinline__ bool next(const int32_t *) { return ++q < q1; }
    };
    using Cur = std::conditional_t<CELLS == 32, CurOne, CurMulti>;
    Cur pc;
    if constexpr (CELLS == 32) pc = CurOne{cbase + lane, off[cbase + lane] - 1, off[cbase + lane + 1]};
    else pc = CurMulti{cbase + lane - 32, 0, 0, cbase + CELLS};
    Cur cc = pc;
    bool hp = pc.next(off);
#pragma unroll
    for (int s0 = 0; s0 < ST; ++s0) {
        if (hp) issue(s0, slot(pc.q));
        cp_async_commit();
        hp = hp && pc.next(off);
    }
    int32_t ppos = hp ? slot(pc.q) : 0;
    bool hc = cc.next(off);
    int stage = 0, cur = -1;
    int bown[D], nb[3];
    if constexpr (D == 2) nb[2] = 0;
    unsigned reach = 0u;                          // node tiles (bit dz dy dx) this lane's cells reach
    CellSums<R, D> acc;
    auto open_cell = [&](int c) {                 // a new cell: its base, first node, reach; zero sums
        cur = c;
        int r = cur;
        unsigned hi = 0u;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int ci = r % Gm::T;
            r /= Gm::T;
            bown[a] = org[a] + ci - 1;         // base cell index of the cell's particles
            nb[a] = org[a] + ci + 1;           // its first stencil node
            hi |= (ci + 3 >= Gm::T ? 1u : 0u) << a;
        }
#pragma unroll
        for (int m = 0; m < (1 << D); ++m)
            if ((m & ~hi & ((1u << D) - 1u)) == 0u) reach |= 1u << m;
        acc.zero();
    };
    auto close_cell = [&]() {                     // the cell is done: its 3^D node sums to the grid
        const int sx = P.G_nodes[0], sxy = P.G_nodes[0] * P.G_nodes[1];
        R4<R> *base = Asim + ((int64_t)nb[2] * P.G_nodes[1] + nb[1]) * sx + nb[0];   // nb[2] = 0 in 2D
#pragma unroll
        for (int kk = 0; kk < Gm::STENCIL; ++kk) {
            R4<R> *node = base + (kk % 3) + ((kk / 3) % 3) * sx + (kk / 9) * sxy;
            if constexpr (ADJ) red_add4(node, acc.q(kk, 0), acc.q(kk, 1), acc.q(kk, 2), R(0));   // (v_bar, 0)
            else red_add4(node, acc.m(kk), acc.q(kk, 0), acc.q(kk, 1), acc.q(kk, 2));          // (m, q)
        }
    };
    constexpr bool ONE = CELLS == 32;             // one cell per lane: opened before, closed after the loop
    if (ONE && hc) open_cell(cc.c);
    while (hc) {
        if constexpr (!ONE) {
            if (cc.c != cur) open_cell(cc.c);
        }
        cp_async_wait<ST - 1>();
        P2GFactors<R, D> f;
        {
            const R *src = stg + stage * NCM * NT + tid;
            if constexpr (ADJ) {
                adj_scatter_factors<R>(P, [&](int j) { return src[j * NT]; }, f);
            } else {
                if (Sv != nullptr) {               // the adjoint's copy of this step's state
                    R *d = Sv + slot(cc.q);
#pragma unroll
                    for (int j = 0; j < NC; ++j) d[j * P.n] = src[j * NT];
                }
                p2g_factors<R, D, MAT>(P, [&](int j) { return src[j * NT]; }, f);
            }
        }
        if (hp) issue(stage, ppos);
        cp_async_commit();
        hp = hp && pc.next(off);
        if (hp) ppos = slot(pc.q);
        bool own = true;
#pragma unroll
        for (int a = 0; a < D; ++a) own = own && (f.b[a] == bown[a]);
        if (own) {
            acc.add(f, mass);
        } else {                                   // left its cell since the sort: on its own
            any_escape = true;
            p2g_escape<R, D>(f, mass, Asim, P.G_nodes[0], P.G_nodes[1], ADJ ? nullptr : io.flags,
                             (int64_t)sim * P.node_tiles_per_sim, P.node_list, P.list_count, P.node_tiles[0],
                             P.node_tiles[1]);
        }
        stage = stage + 1 == ST ? 0 : stage + 1;
        hc = cc.next(off);
        if constexpr (!ONE) {
            if (!hc || cc.c != cur) close_cell();
        }
    }
    if (ONE && cur >= 0) close_cell();
    cp_async_wait<0>();
    if constexpr (!ADJ) {                          // node tiles reached by the warp's cells
        const unsigned wreach = __reduce_or_sync(0xffffffffu, reach);
        if (lane < (1 << D) && ((wreach >> lane) & 1u)) {
            int u[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < D; ++a) u[a] = org[a] / Gm::T + ((lane >> a) & 1);
            mark_node_tile(io.flags, P.node_list, P.list_count,
                           (int64_t)sim * P.node_tiles_per_sim + lin3<D>(u, P.node_tiles));
        }
    }
}

// Resident 128-thread blocks per SM of the 2D cell-ordered P2G.
#ifndef MPM_P2G2_MINB
#define MPM_P2G2_MINB 4
#endif
template <class R, int D, int NT, int MAT>
__global__ void __launch_bounds__(NT, D == 3 ? MPM_P2G_MINB : MPM_P2G2_MINB)
    k_p2g_direct(const Params<R> P, const P2GIO<R> io, unsigned long long *__restrict__ escaped_count,
                 int32_t *__restrict__ g2p_cursor)
{
    using Gm = Geo<D>;
    constexpr int NCM = direct_stage_comps<D, MAT>();
    constexpr int CELLS = direct_cells<D>();         // cells per work item
    constexpr int ITEMS = Gm::TN / CELLS;            // work items per tile
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *stg = reinterpret_cast<R *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31;
    int32_t *const s_off = reinterpret_cast<int32_t *>(smem_raw + (size_t)direct_stages<D>() * NCM * NT * sizeof(R)) +
                           (tid >> 5) * kDirectOffPad;
    const int n_items = *io.n_tiles * ITEMS;
    bool any_escape = false;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(io.cursor, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        const int k = item / ITEMS;
        p2g_direct_item<R, D, NT, MAT>(P, io, stg, s_off, k, (item - k * ITEMS) * CELLS, any_escape);
    }
    if (escaped_count != nullptr) {
        const unsigned ball = __ballot_sync(0xffffffffu, any_escape);
        if (ball && lane == 0) atomicAdd(escaped_count, (unsigned long long)__popc(ball));
    }
    if (g2p_cursor != nullptr && threadIdx.x == 0) *g2p_cursor = 0;   // G2P cursor for the next kernel
}

// ------------------------------------------------------------------ grid update

// Frictionless contact with the stationary obstacles (Sec. 4.1): a node inside a
// box takes the outward normal n of the nearest contact face and, moving into the
// box (v . n < 0), loses its normal component.  The normals are axis-aligned, so
// that component is one coordinate.  Returns the axes it zeroed (bit a).
template <class R, int D>
__device__ __forceinline__ unsigned obstacle_contact(const Params<R> &P, const int a3[3], R vel[3])
{
    unsigned removed = 0u;
    for (int o = 0; o < P.obs.n; ++o) {
        int c[3] = {0, 0, 0};
        bool in = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            c[a] = a3[a] - 2;
            in = in && c[a] >= P.obs.lo[o][a] && c[a] <= P.obs.hi[o][a];
        }
        if (!in) continue;
        const int faces = P.obs.faces[o];
        int best = -1, bd = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int dl = c[a] - P.obs.lo[o][a], dh = P.obs.hi[o][a] - c[a];
            if (((faces >> (2 * a)) & 1) && (best < 0 || dl < bd)) { best = 2 * a; bd = dl; }
            if (((faces >> (2 * a + 1)) & 1) && (best < 0 || dh < bd)) { best = 2 * a + 1; bd = dh; }
        }
        if (best < 0) continue;
        const int ax = best >> 1;
        const bool into = (best & 1) ? vel[ax] < R(0) : vel[ax] > R(0);
        if (into) {
            vel[ax] = R(0);
            removed |= 1u << ax;
        }
    }
    return removed;
}

// Blocks walk the list of node tiles the last P2G touched.
// Reads (m, q + dt f), writes the contact-corrected velocity and clears the
// accumulator for the next step.
template <class R, int D>
__global__ void __launch_bounds__(256) k_grid(const Params<R> P, R4<R> *__restrict__ A,
                                              R4<R> *__restrict__ V, uint32_t *__restrict__ flags,
                                              R4<R> *__restrict__ saveA, R4<R> *__restrict__ saveV,
                                              int32_t *__restrict__ saveL, R4<R> *__restrict__ A2,
                                              R4<R> *__restrict__ V2, const int32_t *__restrict__ list,
                                              const int32_t *__restrict__ count)
{
    using Gm = Geo<D>;
    const int n_list = *count;
    if (saveL != nullptr && blockIdx.x == 0 && threadIdx.x == 0) saveL[0] = n_list;
    // conservation sums (P.diag set): mass, momentum (q + dt f), non-finite values, sum of |q|
    double dsum[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int li = blockIdx.x; li < n_list; li += gridDim.x) {
    const int64_t ut = list[li];
    if (saveL != nullptr && threadIdx.x == 0) saveL[1 + li] = (int32_t)ut;
    const int sim = (int)(ut / P.node_tiles_per_sim);
    int64_t r = ut - (int64_t)sim * P.node_tiles_per_sim;
    int u[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        u[a] = (int)(r % P.node_tiles[a]);
        r /= P.node_tiles[a];
    }
    R4<R> *As = A + (int64_t)sim * P.nodes_per_sim;
    R4<R> *Vs = V + (int64_t)sim * P.nodes_per_sim;
    constexpr int floor_w = 2 * (D - 1);
    for (int i = threadIdx.x; i < Gm::TN; i += blockDim.x) {
        int a3[3] = {0, 0, 0};
        int rr = i;
        bool ok = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            a3[a] = u[a] * Gm::T + rr % Gm::T;
            rr /= Gm::T;
            ok = ok && a3[a] < P.G_nodes[a];
        }
        if (!ok) continue;
        const int64_t idx = lin3<D>(a3, P.G_nodes);
        const R4<R> acc = As[idx];
        if (acc.x == R(0) && acc.y == R(0) && acc.z == R(0) && acc.w == R(0)) continue;
        As[idx] = R4<R>{R(0), R(0), R(0), R(0)};
        if (P.diag != nullptr) {
            dsum[0] += (double)acc.x;
            dsum[1] += (double)acc.y;
            dsum[2] += (double)acc.z;
            dsum[3] += (double)acc.w;
            dsum[4] += (rfinite(acc.x) && rfinite(acc.y) && rfinite(acc.z) && rfinite(acc.w)) ? 0.0 : 1.0;
            dsum[5] += fabs((double)acc.y) + fabs((double)acc.z) + fabs((double)acc.w);
        }
        R vel[3] = {R(0), R(0), R(0)};
        if (acc.x > P.m_eps) {
            const R inv_m = R(1) / acc.x;
            vel[0] = acc.y * inv_m + P.dt * P.gravity[0];
            vel[1] = acc.z * inv_m + P.dt * P.gravity[1];
            if (D == 3) vel[2] = acc.w * inv_m + P.dt * P.gravity[2];
        }
        obstacle_contact<R, D>(P, a3, vel);
        // walls x-, x+, y-, y+, (z-, z+), floor last
#pragma unroll
        for (int q = 0; q < 2 * D; ++q) {
            const int w = q < 2 * D - 1 ? (q < floor_w ? q : q + 1) : floor_w;
            const int ax = w >> 1, hi = w & 1;
            const int c = a3[ax] - 2;
            const bool on = hi ? (c >= P.n_cells[ax]) : (c <= 0);
            if (!on) continue;
            const R vn = hi ? vel[ax] : -vel[ax];
            if (!(vn > R(0))) continue;
            const R mu = wall_mu<R, D>(P, w, sim, a3);
            vel[ax] = R(0);
            if (mu > R(0)) {
                R vt2 = R(0);
#pragma unroll
                for (int bb = 0; bb < D; ++bb) vt2 += vel[bb] * vel[bb];
                const R vt = rsqrt_(vt2);
                const R scale = (vt <= mu * vn) ? R(0) : R(1) - mu * vn / vt;
#pragma unroll
                for (int bb = 0; bb < D; ++bb) vel[bb] *= scale;
            }
        }
        Vs[idx] = R4<R>{vel[0], vel[1], vel[2], R(0)};
        if (A2 != nullptr) {                     // FLIP: grid velocity before the update, v_i^n = q_i / m_i
            const int64_t j2 = (int64_t)sim * P.nodes_per_sim + idx;
            const R4<R> a2 = A2[j2];
            A2[j2] = R4<R>{R(0), R(0), R(0), R(0)};
            const R im = a2.x > P.m_eps ? R(1) / a2.x : R(0);
            V2[j2] = R4<R>{a2.y * im, a2.z * im, a2.w * im, R(0)};
        }
        if (saveA != nullptr) {                  // forward grid kept for the reverse sweep
            saveA[(int64_t)sim * P.nodes_per_sim + idx] = acc;
            saveV[(int64_t)sim * P.nodes_per_sim + idx] = R4<R>{vel[0], vel[1], vel[2], R(0)};
        }
    }
    if (threadIdx.x == 0) flags[ut] = 0u;
    }
    if (P.diag != nullptr) {
        constexpr int slots[6] = {kDiagGridMass, kDiagGridMom, kDiagGridMom + 1, kDiagGridMom + 2, kDiagGridNonFinite,
                                  kDiagGridAbsMom};
        block_sum_add<6>(dsum, P.diag, slots);
    }
}

// Conservation sums of the particles the next P2G reads (P.diag set): total mass,
// momentum sum m_p v_p and the count of particles with a non-finite x or v.
template <class R, int D>
__global__ void __launch_bounds__(256) k_diag_particles(const Params<R> P, const R *__restrict__ S)
{
    double dsum[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const double mp = (double)P.mass;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P.n; p += (int64_t)gridDim.x * blockDim.x) {
        bool fin = true;
        dsum[0] += mp;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const R v = S[sblock(p, P.ncomp) + (P.off_v + a) * kPB];
            const R x = S[sblock(p, P.ncomp) + (P.off_x + a) * kPB];
            fin = fin && rfinite(v) && rfinite(x);
            dsum[1 + a] += mp * (double)v;
        }
        dsum[4] += fin ? 0.0 : 1.0;
    }
    constexpr int slots[5] = {kDiagPartMass, kDiagPartMom, kDiagPartMom + 1, kDiagPartMom + 2, kDiagPartNonFinite};
    block_sum_add<5>(dsum, P.diag, slots);
}

// ------------------------------------------------------------------ G2P

// Drucker-Prager update of Appendix A in symmetric storage (xx, yy, zz, xy,
// xz, yz).  L is the 3 x 3 velocity gradient (zero third row/column in 2D).
template <class R>
__device__ __forceinline__ void dp_update(const Params<R> &P, const R L[9], R s[6], R &eps)
{
    const R dt = P.dt;
    const R d0 = dt * L[0], d1 = dt * L[4], d2 = dt * L[8];
    const R d3 = R(0.5) * dt * (L[1] + L[3]);
    const R d4 = R(0.5) * dt * (L[2] + L[6]);
    const R d5 = R(0.5) * dt * (L[5] + L[7]);
    const R w01 = R(0.5) * dt * (L[1] - L[3]);
    const R w02 = R(0.5) * dt * (L[2] - L[6]);
    const R w12 = R(0.5) * dt * (L[5] - L[7]);
    // full stress and spin W (W_01 = w01, W_02 = w02, W_12 = w12, antisymmetric)
    const R S00 = s[0], S11 = s[1], S22 = s[2], S01 = s[3], S02 = s[4], S12 = s[5];
    // M = W S
    const R M00 = w01 * S01 + w02 * S02;
    const R M01 = w01 * S11 + w02 * S12;
    const R M02 = w01 * S12 + w02 * S22;
    const R M10 = -w01 * S00 + w12 * S02;
    const R M11 = -w01 * S01 + w12 * S12;
    const R M12 = -w01 * S02 + w12 * S22;
    const R M20 = -w02 * S00 - w12 * S01;
    const R M21 = -w02 * S01 - w12 * S11;
    const R M22 = -w02 * S02 - w12 * S12;
    // rotated stress S + M + M^T, then trial stress with isotropic elasticity
    const R lam_tr = (P.K - R(2) / R(3) * P.G) * (d0 + d1 + d2);
    const R twoG = R(2) * P.G;
    R t[6];
    t[0] = S00 + R(2) * M00 + lam_tr + twoG * d0;
    t[1] = S11 + R(2) * M11 + lam_tr + twoG * d1;
    t[2] = S22 + R(2) * M22 + lam_tr + twoG * d2;
    t[3] = S01 + M01 + M10 + twoG * d3;
    t[4] = S02 + M02 + M20 + twoG * d4;
    t[5] = S12 + M12 + M21 + twoG * d5;
    const R sm = (t[0] + t[1] + t[2]) * R(1.0 / 3.0);     // the mean stress (a product: no divide)
    R dev[6] = {t[0] - sm, t[1] - sm, t[2] - sm, t[3], t[4], t[5]};
    const R tau = rsqrt_(R(0.5) * (dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2]) +
                         dev[3] * dev[3] + dev[4] * dev[4] + dev[5] * dev[5]);
    const R fs = tau - P.k_phi + P.q_phi * sm;
    const R ft = sm - P.sig_t;
    const R h = tau - P.tau_P - P.alpha_P * (sm - P.sig_t);
    if (fs <= R(0) && ft < R(0)) {
#pragma unroll
        for (int k = 0; k < 6; ++k) s[k] = t[k];
        return;
    }
    if ((fs > R(0) && ft < R(0)) || (h > R(0) && ft >= R(0))) {
        const R dl = fs * P.inv_G_Kqq;                 // fs / (G + K q_phi q_psi)
        R smn = sm - P.K * P.q_psi * dl;
        R taun = P.k_phi - P.q_phi * smn;
        if (!P.dp_literal && smn > P.sig_t) {
            smn = P.sig_t;
            taun = P.tau_P;
        }
        const R r = tau > R(0) ? taun / tau : R(0);
        s[0] = r * dev[0] + smn; s[1] = r * dev[1] + smn; s[2] = r * dev[2] + smn;
        s[3] = r * dev[3]; s[4] = r * dev[4]; s[5] = r * dev[5];
        eps += dl * P.eps2_coef;
        return;
    }
    eps += (sm - P.sig_t) * P.inv_K * (R(1.4142135623730951) / R(3));
    R r = R(1);
    if (!P.dp_literal && tau > P.tau_P) r = P.tau_P / tau;
    s[0] = r * dev[0] + P.sig_t; s[1] = r * dev[1] + P.sig_t; s[2] = r * dev[2] + P.sig_t;
    s[3] = r * dev[3]; s[4] = r * dev[4]; s[5] = r * dev[5];
}

// Separable G2P sums over the 3^D stencil: with tensor-product weights
//   vp_a = sum w v_a,  M_ab = sum w v_a k_b,  L_ab = sum (grad w)_b v_a,
// contracted one axis at a time (x, then y, then z).
template <class R, int D, class Load>
__device__ __forceinline__ void g2p_contract(const R w[D][3], const R dw[D][3], Load load, R vp[D], R M[D * D],
                                             R L[D * D])
{
#pragma unroll
    for (int q = 0; q < D; ++q) vp[q] = R(0);
#pragma unroll
    for (int q = 0; q < D * D; ++q) {
        M[q] = R(0);
        L[q] = R(0);
    }
    if constexpr (D == 2) {
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            R Xw[2] = {R(0), R(0)}, Xk[2] = {R(0), R(0)}, Xd[2] = {R(0), R(0)};
#pragma unroll
            for (int k0 = 0; k0 < 3; ++k0) {
                const R4<R> v4 = load(k0, k1, 0);
                const R v[2] = {v4.x, v4.y};
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    Xw[a] = fma(w[0][k0], v[a], Xw[a]);
                    if (k0 > 0) Xk[a] = fma(R(k0) * w[0][k0], v[a], Xk[a]);
                    Xd[a] = fma(dw[0][k0], v[a], Xd[a]);
                }
            }
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                vp[a] = fma(w[1][k1], Xw[a], vp[a]);
                M[a * 2 + 0] = fma(w[1][k1], Xk[a], M[a * 2 + 0]);
                if (k1 > 0) M[a * 2 + 1] = fma(R(k1) * w[1][k1], Xw[a], M[a * 2 + 1]);
                L[a * 2 + 0] = fma(w[1][k1], Xd[a], L[a * 2 + 0]);
                L[a * 2 + 1] = fma(dw[1][k1], Xw[a], L[a * 2 + 1]);
            }
        }
    } else {
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2) {
            R Yww[3], Ykw[3], Ydw[3], Ywk[3], Ywd[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) Yww[a] = Ykw[a] = Ydw[a] = Ywk[a] = Ywd[a] = R(0);
#pragma unroll
            for (int k1 = 0; k1 < 3; ++k1) {
                R Xw[3], Xk[3], Xd[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) Xw[a] = Xk[a] = Xd[a] = R(0);
#pragma unroll
                for (int k0 = 0; k0 < 3; ++k0) {
                    const R4<R> v4 = load(k0, k1, k2);
                    const R v[3] = {v4.x, v4.y, v4.z};
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        Xw[a] = fma(w[0][k0], v[a], Xw[a]);
                        if (k0 > 0) Xk[a] = fma(R(k0) * w[0][k0], v[a], Xk[a]);
                        Xd[a] = fma(dw[0][k0], v[a], Xd[a]);
                    }
                }
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Yww[a] = fma(w[1][k1], Xw[a], Yww[a]);
                    Ykw[a] = fma(w[1][k1], Xk[a], Ykw[a]);
                    Ydw[a] = fma(w[1][k1], Xd[a], Ydw[a]);
                    if (k1 > 0) Ywk[a] = fma(R(k1) * w[1][k1], Xw[a], Ywk[a]);
                    Ywd[a] = fma(dw[1][k1], Xw[a], Ywd[a]);
                }
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                vp[a] = fma(w[2][k2], Yww[a], vp[a]);
                M[a * 3 + 0] = fma(w[2][k2], Ykw[a], M[a * 3 + 0]);
                M[a * 3 + 1] = fma(w[2][k2], Ywk[a], M[a * 3 + 1]);
                if (k2 > 0) M[a * 3 + 2] = fma(R(k2) * w[2][k2], Yww[a], M[a * 3 + 2]);
                L[a * 3 + 0] = fma(w[2][k2], Ydw[a], L[a * 3 + 0]);
                L[a * 3 + 1] = fma(w[2][k2], Ywd[a], L[a * 3 + 1]);
                L[a * 3 + 2] = fma(dw[2][k2], Yww[a], L[a * 3 + 2]);
            }
        }
    }
}

// The same sums in single precision in 3D with paired arithmetic: the x and y
// components of a node velocity are adjacent (the low half of its 16-byte
// load), so the sums of components 0 and 1 run as one paired fused multiply-add
// (__ffma2_rn, each half rounded as fmaf) against a weight broadcast into both
// halves; component 2 stays scalar.  The results are bitwise those of the
// scalar form above, in about two thirds of the instructions.
template <class Load>
__device__ __forceinline__ void g2p_contract_x2(const float w[3][3], const float dw[3][3], Load load, float vp[3],
                                                float M[9], float L[9])
{
    auto bc = [](float a) { return make_float2(a, a); };
    float2 vp01 = make_float2(0.f, 0.f), M01[3], L01[3];
    float vp2 = 0.f, M2[3] = {0.f, 0.f, 0.f}, L2[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < 3; ++b) M01[b] = L01[b] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2) {
        float2 Yww = make_float2(0.f, 0.f), Ykw = Yww, Ydw = Yww, Ywk = Yww, Ywd = Yww;
        float yww = 0.f, ykw = 0.f, ydw = 0.f, ywk = 0.f, ywd = 0.f;
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            float2 Xw = make_float2(0.f, 0.f), Xk = Xw, Xd = Xw;
            float xw = 0.f, xk = 0.f, xd = 0.f;
#pragma unroll
            for (int k0 = 0; k0 < 3; ++k0) {
                const R4<float> v4 = load(k0, k1, k2);
                const float2 v01 = make_float2(v4.x, v4.y);
                Xw = __ffma2_rn(bc(w[0][k0]), v01, Xw);
                xw = fmaf(w[0][k0], v4.z, xw);
                if (k0 > 0) {
                    Xk = __ffma2_rn(bc(float(k0) * w[0][k0]), v01, Xk);
                    xk = fmaf(float(k0) * w[0][k0], v4.z, xk);
                }
                Xd = __ffma2_rn(bc(dw[0][k0]), v01, Xd);
                xd = fmaf(dw[0][k0], v4.z, xd);
            }
            Yww = __ffma2_rn(bc(w[1][k1]), Xw, Yww);
            yww = fmaf(w[1][k1], xw, yww);
            Ykw = __ffma2_rn(bc(w[1][k1]), Xk, Ykw);
            ykw = fmaf(w[1][k1], xk, ykw);
            Ydw = __ffma2_rn(bc(w[1][k1]), Xd, Ydw);
            ydw = fmaf(w[1][k1], xd, ydw);
            if (k1 > 0) {
                Ywk = __ffma2_rn(bc(float(k1) * w[1][k1]), Xw, Ywk);
                ywk = fmaf(float(k1) * w[1][k1], xw, ywk);
            }
            Ywd = __ffma2_rn(bc(dw[1][k1]), Xw, Ywd);
            ywd = fmaf(dw[1][k1], xw, ywd);
        }
        vp01 = __ffma2_rn(bc(w[2][k2]), Yww, vp01);
        vp2 = fmaf(w[2][k2], yww, vp2);
        M01[0] = __ffma2_rn(bc(w[2][k2]), Ykw, M01[0]);
        M2[0] = fmaf(w[2][k2], ykw, M2[0]);
        M01[1] = __ffma2_rn(bc(w[2][k2]), Ywk, M01[1]);
        M2[1] = fmaf(w[2][k2], ywk, M2[1]);
        if (k2 > 0) {
            M01[2] = __ffma2_rn(bc(float(k2) * w[2][k2]), Yww, M01[2]);
            M2[2] = fmaf(float(k2) * w[2][k2], yww, M2[2]);
        }
        L01[0] = __ffma2_rn(bc(w[2][k2]), Ydw, L01[0]);
        L2[0] = fmaf(w[2][k2], ydw, L2[0]);
        L01[1] = __ffma2_rn(bc(w[2][k2]), Ywd, L01[1]);
        L2[1] = fmaf(w[2][k2], ywd, L2[1]);
        L01[2] = __ffma2_rn(bc(dw[2][k2]), Yww, L01[2]);
        L2[2] = fmaf(dw[2][k2], yww, L2[2]);
    }
    vp[0] = vp01.x;
    vp[1] = vp01.y;
    vp[2] = vp2;
#pragma unroll
    for (int b = 0; b < 3; ++b) {           // M[a * 3 + b], L[a * 3 + b]; the pairs run over a
        M[0 * 3 + b] = M01[b].x;
        M[1 * 3 + b] = M01[b].y;
        M[2 * 3 + b] = M2[b];
        L[0 * 3 + b] = L01[b].x;
        L[1 * 3 + b] = L01[b].y;
        L[2 * 3 + b] = L2[b];
    }
}

#ifndef MPM_G2P_X2
#define MPM_G2P_X2 1
#endif

// G2P of one particle: gathers the 3^D node velocities from the shared-memory
// window (or from the global grid if its stencil left the window), then
// updates v, C, x, F, rho and the stress.  Returns false on a non-finite state.
// Components of the particle state G2P reads, in staging order: x (D), F (D^2),
// rho, and for Drucker-Prager sigma (6) and eps.  rho, sigma, eps are consecutive.
template <int D> __host__ __device__ __forceinline__ constexpr int g2p_ncomp(int material)
{
    return D + D * D + 1 + (material == 1 ? 7 : 0);
}


template <class R, int D, bool GENERIC, int MAT, class Raw>
__device__ __forceinline__ bool g2p_particle(const Params<R> &P, Raw raw, R *__restrict__ S, int64_t p,
                                             const R4<R> *Vw, const int org[3], const R4<R> *__restrict__ Vs,
                                             const R4<R> *__restrict__ V2s = nullptr)
{
    using Gm = Geo<D>;
    using Ly = Lay<D, MAT>;
    constexpr int J_F = D, J_RHO = D + D * D;
    constexpr int64_t np = kPB;                    // component stride inside a particle block
    R *__restrict__ Sp = S + sblock(p, Ly::NC);    // component c of this particle at Sp[c kPB]
    bool bad = false;
    R x[D];
#pragma unroll
    for (int a = 0; a < D; ++a) x[a] = raw(a);
    int b[D], l[D];
    R fx[D], w[D][3], dw[D][3];
    bool inside = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        b[a] = base_cell(x[a], P.inv_dx, P.n_cells[a]);
        fx[a] = x[a] * P.inv_dx - R(b[a]);
        bspline(fx[a], P.inv_dx, w[a], dw[a]);
        l[a] = b[a] + 2 - org[a];
        inside = inside && l[a] >= 0 && l[a] <= Gm::W - 3;
    }
    R vp[D], M[D * D], L[D * D];
    if (inside) {
        if constexpr (D == 3 && sizeof(R) == 4 && MPM_G2P_X2)
            g2p_contract_x2(w, dw, [&](int k0, int k1, int k2) { return Vw[win_index<D>(l, k0, k1, k2)]; }, vp, M,
                            L);
        else
            g2p_contract<R, D>(w, dw, [&](int k0, int k1, int k2) { return Vw[win_index<D>(l, k0, k1, k2)]; }, vp, M,
                               L);
    } else {
        g2p_contract<R, D>(w, dw, [&](int k0, int k1, int k2) {
            int a3[3] = {b[0] + 2 + k0, b[1] + 2 + k1, D == 3 ? b[D - 1] + 2 + k2 : 0};
            return Vs[lin3<D>(a3, P.G_nodes)];
        }, vp, M, L);
    }
    // B_ab = sum w v_a (k_b - fx_b) (units of dx) = M_ab - fx_b vp_a
    R Bm[D * D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c2 = 0; c2 < D; ++c2) Bm[a * D + c2] = M[a * D + c2] - fx[c2] * vp[a];
    // C = B D^{-1} with D = dx^2 / 4 I; B was accumulated in units of dx
    const R cscale = R(4) * P.inv_dx;
    R trL = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) trL += L[a * D + a];
    // FLIP / PIC blend: v_p = v_PIC + alpha (v_p - sum w v_i^n)
    R vnew[D];
#pragma unroll
    for (int a = 0; a < D; ++a) vnew[a] = vp[a];
    if (GENERIC && P.transfer == 3) {
        R vo[D];
#pragma unroll
        for (int a = 0; a < D; ++a) vo[a] = R(0);
#pragma unroll
        for (int k = 0; k < Gm::STENCIL; ++k) {
            const int kk[3] = {k % 3, (k / 3) % 3, k / 9};
            R wk = R(1);
            int a3[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < D; ++a) {
                wk *= w[a][kk[a]];
                a3[a] = b[a] + 2 + kk[a];
            }
            const R4<R> v4 = V2s[lin3<D>(a3, P.G_nodes)];
            const R vi[3] = {v4.x, v4.y, v4.z};
#pragma unroll
            for (int a = 0; a < D; ++a) vo[a] += wk * vi[a];
        }
#pragma unroll
        for (int a = 0; a < D; ++a) vnew[a] = vp[a] + P.flip_alpha * (Sp[(Ly::V + a) * np] - vo[a]);
    }
    // one finiteness test for the whole new state: a sum of finite values is finite
    // (values near the overflow threshold are themselves a blown-up state), and a
    // non-finite term makes it +-inf or NaN
    R chk = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        R xn = x[a] + P.dt * vp[a];
        xn = xn < R(0) ? R(0) : (xn > P.L[a] ? P.L[a] : xn);
        chk += xn + vnew[a];
        Sp[(Ly::X + a) * np] = xn;
        Sp[(Ly::V + a) * np] = vnew[a];
    }
    // particle matrix for the next P2G: APIC C = B D^-1, TPIC the velocity gradient, PIC none
#pragma unroll
    for (int q = 0; q < D * D; ++q)
        Sp[(Ly::C + q) * np] = !GENERIC ? Bm[q] * cscale
                                        : (P.transfer == 1 ? L[q] : (P.transfer >= 2 ? R(0) : Bm[q] * cscale));
    // F <- (I + dt L) F
    R F[D * D];
#pragma unroll
    for (int q = 0; q < D * D; ++q) F[q] = raw(J_F + q);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c2 = 0; c2 < D; ++c2) {
            R s = R(0);
#pragma unroll
            for (int k = 0; k < D; ++k) s += L[a * D + k] * F[k * D + c2];
            Sp[(Ly::F + a * D + c2) * np] = F[a * D + c2] + P.dt * s;
        }
    const R rho = raw(J_RHO) / (R(1) + P.dt * trL);
    Sp[Ly::RHO * np] = rho;
    chk += rho;
    if constexpr (MAT == 1) {
        R L3[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) L3[q] = R(0);
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int c2 = 0; c2 < D; ++c2) L3[a * 3 + c2] = L[a * D + c2];
        R s6[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) s6[k] = raw(J_RHO + 1 + k);
        R e = raw(J_RHO + 7);
        dp_update(P, L3, s6, e);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            Sp[(Ly::SIG + k) * np] = s6[k];
            chk += s6[k];
        }
        Sp[Ly::EPS * np] = e;
    }
    return !bad && rfinite(chk);
}

// Shared-memory layout of the G2P block: the grid window, then two staging
// buffers of NT / kPB particle blocks (the components G2P reads).
// Particles per thread in one staged chunk of the G2P block (3D, 2D): chunks of 512
// particles halve the block barriers per particle (3D dam break G2P 0.071 -> 0.067
// ms, 2D batched 0.080 -> 0.074 ms; the 2.76M-particle collapse 0.118 -> 0.116).
#ifndef MPM_G2P_PPT
#define MPM_G2P_PPT 2
#endif
#ifndef MPM_G2P2_PPT
#define MPM_G2P2_PPT 2
#endif
template <class R, int D> struct G2PSmem {
    static constexpr int NT = 256;
    static constexpr int CH = NT * (sizeof(R) == 4 ? (D == 3 ? MPM_G2P_PPT : MPM_G2P2_PPT) : 1);   // per chunk
    static constexpr int NBLK = CH / kPB;
    static constexpr int NCMAX = D + D * D + 8;
    static constexpr size_t win_bytes = (size_t)Geo<D>::WN * sizeof(R4<R>);
    static constexpr size_t buf_elems = (size_t)NBLK * NCMAX * kPB;
    static constexpr size_t buf_bytes = 2 * buf_elems * sizeof(R);
    static constexpr size_t total = win_bytes + buf_bytes + 128;
};

// G2P of one tile t (compact list entry) by a block of NT threads: the tile's
// velocity window by one TMA tensor copy, the particles in chunks of CH slots
// aligned to the particle blocks, staged by bulk copies into two buffers of
// buf_elems reals.  Returns false when a bounded wait ran out.
template <class R, int D, bool GENERIC, int MAT, int NT, int CH>
__device__ __forceinline__ bool g2p_tile(const Params<R> &P, const CUtensorMap *tmapV, R *__restrict__ S,
                                         const R4<R> *__restrict__ V, const R4<R> *__restrict__ V2, int4 t,
                                         R4<R> *Vw, R *bufs, size_t buf_elems, uint64_t *mbar, uint32_t &phases,
                                         bool &bad)
{
    using Gm = Geo<D>;
    using Ly = Lay<D, MAT>;
    constexpr int nc = Ly::G2P_IN;
    const int tid = threadIdx.x;
    const int sim = (int)(t.x / P.tiles_per_sim);
    int64_t tl = t.x - (int64_t)sim * P.tiles_per_sim;
    int org[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        org[a] = (int)(tl % P.n_tiles[a]) * Gm::T;
        tl /= P.n_tiles[a];
    }
    if (tid == 0 && !(P.debug & kDebugWithholdWindowCopy)) {
        fence_proxy_async_smem();
        mbar_expect_tx(&mbar[2], (uint32_t)(Gm::WN * sizeof(R4<R>)));
        tma_load_window(Vw, tmapV, org, sim, D, &mbar[2]);
    }
    // particles in chunks of CH slots aligned to the particle blocks (so a warp's
    // 32 particles are one block and each of its stores writes one line); slots
    // of a neighbouring tile at either end are skipped
    const int64_t a0 = (int64_t)t.y & ~(int64_t)(kPB - 1);
    const int64_t pend = (int64_t)t.y + t.z;
    const int nb = (int)((pend - a0 + CH - 1) / CH);
    int cur = 0;
    stage_blocks(bufs, S, Ly::NC, nc, a0, (int)(pend - a0 < CH ? pend - a0 : CH), &mbar[0]);
    bool ok = mbar_wait_bounded(&mbar[2], (phases >> 2) & 1u);
    phases ^= 4u;
    const R4<R> *Vs = V + (int64_t)sim * P.nodes_per_sim;
    const R4<R> *V2s = V2 != nullptr ? V2 + (int64_t)sim * P.nodes_per_sim : nullptr;
    for (int j = 0; j < nb; ++j) {
        if (j + 1 < nb) {
            const int64_t an = a0 + (int64_t)(j + 1) * CH;
            stage_blocks(bufs + (size_t)(cur ^ 1) * buf_elems, S, Ly::NC, nc, an,
                         (int)(pend - an < CH ? pend - an : CH), &mbar[cur ^ 1]);
        }
        const bool okb = mbar_wait_bounded(&mbar[cur], (phases >> cur) & 1u);
        phases ^= 1u << cur;
        ok = ok && okb;
#pragma unroll 1
        for (int u = 0; u < CH / NT; ++u) {
            const int l = u * NT + tid;                // slot within the chunk
            const int64_t p = a0 + (int64_t)j * CH + l;
            if (ok && p >= t.y && p < pend) {
                const R *bb = bufs + (size_t)cur * buf_elems + (l >> 5) * (nc * kPB) + (l & (kPB - 1));
                bad |= !g2p_particle<R, D, GENERIC, MAT>(P, [&](int jj) { return bb[jj * kPB]; }, S, p, Vw, org,
                                                        Vs, V2s);
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    return ok;
}

// G2P.  Blocks claim tiles dynamically, one thread per particle.  The tile's
// grid window of velocities is staged by one TMA tiled load; the particles'
// inputs are staged 256 at a time by TMA bulk copies, double-buffered.  All
// waits are bounded; a timeout is reported in the status word.
template <class R, int D, bool GENERIC, int MAT>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? MPM_G2P_MINB : 1)
    k_g2p(const Params<R> P, const __grid_constant__ CUtensorMap tmapV, R *__restrict__ S,
          const R4<R> *__restrict__ V, const int4 *__restrict__ tiles, int32_t *__restrict__ counters,
          int32_t *__restrict__ status, const R4<R> *__restrict__ V2)
{
    using Gm = Geo<D>;
    using L = G2PSmem<R, D>;
    constexpr int NT = L::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // 128-byte aligned start for the TMA window, by pointer arithmetic on the shared
    // array (an integer round trip would hide the address space from the compiler and
    // turn every shared access into a generic one)
    unsigned char *base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    R4<R> *Vw = reinterpret_cast<R4<R> *>(base);
    R *bufs = reinterpret_cast<R *>(base + L::win_bytes);
    __shared__ __align__(8) uint64_t mbar[3];      // [0], [1]: particle buffers, [2]: grid window
    __shared__ int s_slot;
    const int tid = threadIdx.x;
    using Ly = Lay<D, MAT>;
    constexpr int nc = Ly::G2P_IN;                 // x, F, rho [, sigma, eps]: the first nc components
    static_assert(nc == g2p_ncomp<D>(MAT), "G2P inputs lead the particle state");
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_init(&mbar[2], 1);
        fence_mbar_init();
    }
    uint32_t phases = 0u;                          // bit i: parity of the next wait on mbar[i]
    bool bad = false, timed_out = false;
    const int n_tiles = counters[1];
    for (;;) {
        const int k = next_tile(&counters[3], n_tiles, &s_slot);
        if (k < 0) break;
        const int4 t = tiles[k];
        const bool ok = g2p_tile<R, D, GENERIC, MAT, NT, L::CH>(P, &tmapV, S, V, V2, t, Vw, bufs, L::buf_elems, mbar,
                                                             phases, bad);
        timed_out |= !ok;
        if (__syncthreads_or(timed_out)) {
            if (tid == 0) atomicOr(status, (int32_t)kStatusTimeout);
            break;
        }
    }
    if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(status, (int32_t)kStatusNaN);
    if (tid == 0) {
        counters[2] = 0;                           // P2G cursor for the next kernel (P2G follows)
        counters[4] = 0;                           // the grid update has walked the touched-tile list
    }
}

// ------------------------------------------------------------------ state management

template <class R, int D>
__global__ void k_init_state(const Params<R> P, R *__restrict__ S, int32_t *__restrict__ id,
                             const double *__restrict__ x, const double *__restrict__ v)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        R *Sp = S + sblock(p, P.ncomp);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            Sp[(P.off_x + a) * kPB] = (R)x[p * D + a];
            Sp[(P.off_v + a) * kPB] = v ? (R)v[p * D + a] : R(0);
        }
#pragma unroll
        for (int q = 0; q < D * D; ++q) {
            Sp[(P.off_C + q) * kPB] = R(0);
            Sp[(P.off_F + q) * kPB] = (q % (D + 1) == 0) ? R(1) : R(0);
        }
        Sp[P.off_rho * kPB] = P.rho0;
        if (P.material == 1) {
            for (int k = 0; k < 6; ++k) Sp[(P.off_sig + k) * kPB] = R(0);
            Sp[P.off_eps * kPB] = R(0);
        }
        id[p] = (int32_t)p;
    }
}

template <class R, int D>
__global__ void k_keys(const Params<R> P, const R *__restrict__ S, const int32_t *__restrict__ sim,
                       uint32_t *__restrict__ keys, int32_t *__restrict__ vals)
{
    using Gm = Geo<D>;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const R *Sp = S + sblock(p, P.ncomp);
        int64_t tile = 0, cell = 0, tstride = 1, cstride = 1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int s = base_cell(Sp[(P.off_x + a) * kPB], P.inv_dx, P.n_cells[a]) + 1;   // [0, N]
            tile += (int64_t)(s / Gm::T) * tstride;
            cell += (int64_t)(s % Gm::T) * cstride;
            tstride *= P.n_tiles[a];
            cstride *= Gm::T;
        }
        const int64_t tkey = (int64_t)sim[p] * P.tiles_per_sim + tile;
        keys[p] = (uint32_t)((tkey << Gm::CELL_BITS) | cell);
        vals[p] = (int32_t)p;
    }
}

template <class R>
__global__ void k_permute(int ncomp, int64_t n, int64_t npad, const R *__restrict__ S, R *__restrict__ S2,
                          const int32_t *__restrict__ perm, const int32_t *__restrict__ id,
                          int32_t *__restrict__ id2, const int32_t *__restrict__ sim,
                          int32_t *__restrict__ sim2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = perm[i];
        o = o < 0 ? 0 : (o >= n ? n - 1 : o);       // defensive: never gather outside the state
        const R *src = S + sblock(o, ncomp);
        R *dst = S2 + sblock(i, ncomp);
        for (int c = 0; c < ncomp; ++c) dst[c * kPB] = src[c * kPB];
        id2[i] = id[o];
        sim2[i] = sim[o];
    }
}

// Field readback in load order (doubles).
template <class R, int D>
__global__ void k_get_field(const Params<R> P, const R *__restrict__ S, const int32_t *__restrict__ id,
                            int field, double *__restrict__ out)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = id[p];
        const R *Sp = S + sblock(p, P.ncomp);
        switch (field) {
        case 0:
            for (int a = 0; a < D; ++a) out[o * D + a] = (double)Sp[(P.off_x + a) * kPB];
            break;
        case 1:
            for (int a = 0; a < D; ++a) out[o * D + a] = (double)Sp[(P.off_v + a) * kPB];
            break;
        case 2:
            for (int q = 0; q < D * D; ++q) out[o * D * D + q] = (double)Sp[(P.off_C + q) * kPB];
            break;
        case 3:
            for (int q = 0; q < D * D; ++q) out[o * D * D + q] = (double)Sp[(P.off_F + q) * kPB];
            break;
        case 4:
            out[o] = (double)Sp[P.off_rho * kPB];
            break;
        case 5: {
            double s9[9];
            if (P.material == 0) {
                const double pr = (double)tait(P, Sp[P.off_rho * kPB]);
                for (int q = 0; q < 9; ++q) s9[q] = (q % 4 == 0) ? -pr : 0.0;
            } else {
                const int map[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};
                for (int q = 0; q < 9; ++q) s9[q] = (double)Sp[(P.off_sig + map[q]) * kPB];
            }
            for (int q = 0; q < 9; ++q) out[o * 9 + q] = s9[q];
            break;
        }
        case 6:
            out[o] = P.material == 1 ? (double)Sp[P.off_eps * kPB] : 0.0;
            break;
        default:
            break;
        }
    }
}

template <class R, int D>
__global__ void k_set_field(const Params<R> P, R *__restrict__ S, const int32_t *__restrict__ id, int field,
                            const double *__restrict__ in)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = id[p];
        R *Sp = S + sblock(p, P.ncomp);
        switch (field) {
        case 0:
            for (int a = 0; a < D; ++a) Sp[(P.off_x + a) * kPB] = (R)in[o * D + a];
            break;
        case 1:
            for (int a = 0; a < D; ++a) Sp[(P.off_v + a) * kPB] = (R)in[o * D + a];
            break;
        case 2:
            for (int q = 0; q < D * D; ++q) Sp[(P.off_C + q) * kPB] = (R)in[o * D * D + q];
            break;
        case 3:
            for (int q = 0; q < D * D; ++q) Sp[(P.off_F + q) * kPB] = (R)in[o * D * D + q];
            break;
        case 4:
            Sp[P.off_rho * kPB] = (R)in[o];
            break;
        case 5: {
            const double *s9 = in + o * 9;
            Sp[(P.off_sig + 0) * kPB] = (R)s9[0];
            Sp[(P.off_sig + 1) * kPB] = (R)s9[4];
            Sp[(P.off_sig + 2) * kPB] = (R)s9[8];
            Sp[(P.off_sig + 3) * kPB] = (R)(0.5 * (s9[1] + s9[3]));
            Sp[(P.off_sig + 4) * kPB] = (R)(0.5 * (s9[2] + s9[6]));
            Sp[(P.off_sig + 5) * kPB] = (R)(0.5 * (s9[5] + s9[7]));
            break;
        }
        case 6:
            Sp[P.off_eps * kPB] = (R)in[o];
            break;
        default:
            break;
        }
    }
}

// ------------------------------------------------------------------ launchers

template <class R>
Params<R> make_params(const HostParams &h, const DevState &ds)
{
    Params<R> P{};
    for (int a = 0; a < 3; ++a) {
        P.n_cells[a] = h.n_cells[a];
        P.gravity[a] = (R)h.gravity[a];
        P.L[a] = (R)(h.n_cells[a] * h.dx);
        P.n_tiles[a] = h.n_tiles[a];
        P.G_nodes[a] = h.G_nodes[a];
        P.node_tiles[a] = h.node_tiles[a];
    }
    P.dx = (R)h.dx;
    P.inv_dx = (R)(1.0 / h.dx);
    P.dt = (R)h.dt;
    P.rho0 = (R)h.rho0;
    P.inv_rho0 = (R)(1.0 / h.rho0);
    P.bulk_K = (R)h.bulk_K;
    P.gamma = (R)h.gamma;
    P.K_over_gamma = (R)(h.bulk_K / h.gamma);
    const double gr = std::floor(h.gamma);
    P.gamma_int = (gr == h.gamma && h.gamma >= 1.0 && h.gamma <= 16.0) ? (int)gr : 0;
    P.mass = (R)h.mass;
    P.m_eps = (R)h.m_eps;
    P.K = (R)h.K; P.G = (R)h.G;
    P.q_phi = (R)h.q_phi; P.k_phi = (R)h.k_phi; P.q_psi = (R)h.q_psi;
    P.sig_t = (R)h.sig_t; P.tau_P = (R)h.tau_P; P.alpha_P = (R)h.alpha_P;
    P.eps2_coef = (R)std::sqrt(1.0 / 3.0 + 2.0 / 9.0 * h.q_psi * h.q_psi);
    P.inv_G_Kqq = h.material == 1 ? (R)(1.0 / (h.G + h.K * h.q_phi * h.q_psi)) : R(0);
    P.inv_K = h.material == 1 ? (R)(1.0 / h.K) : R(0);
    P.material = h.material;
    P.dp_literal = h.dp_literal;
    P.transfer = h.transfer;
    P.flip_alpha = (R)h.flip_alpha;
    P.no_force = 0;
    P.save_S = (R *)ds.save_S;
    P.flags = ds.flags;
    P.node_list = ds.node_list;
    P.list_count = ds.counters + 4;
    P.nodes_per_sim = h.nodes_per_sim;
    P.tiles_per_sim = h.tiles_per_sim;
    P.node_tiles_per_sim = h.node_tiles_per_sim;
    P.n = h.n;
    P.npad = h.npad;
    P.ncomp = h.ncomp;
    P.off_x = h.off_x; P.off_v = h.off_v; P.off_C = h.off_C; P.off_F = h.off_F;
    P.off_rho = h.off_rho; P.off_sig = h.off_sig; P.off_eps = h.off_eps;
    P.obs = h.obs;
    P.diag = ds.diag;
    P.debug = h.debug;
    for (int w = 0; w < kMaxWalls; ++w) {
        P.wall[w].mu = ds.mu_dev[w];
        P.wall[w].n_seg[0] = ds.n_seg[w][0];
        P.wall[w].n_seg[1] = ds.n_seg[w][1];
        int nt = 0;
        for (int b = 0; b < h.dim; ++b)
            if (b != w / 2) P.wall[w].seg_axis[nt++] = b;
        if (nt < 2) P.wall[w].seg_axis[1] = 0;
    }
    return P;
}

inline int grid_blocks(int64_t n, int threads, int num_sms, int per_sm = 16)
{
    int64_t b = (n + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * per_sm;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

template <class R, int D> struct Launch {
    static void init_state(const HostParams &h, DevState &ds, const double *x, const double *v)
    {
        auto P = make_params<R>(h, ds);
        k_init_state<R, D><<<grid_blocks(h.n, 256, ds.num_sms), 256, 0, ds.stream>>>(
            P, (R *)ds.S, ds.id, x, v);
    }
    static void keys(const HostParams &h, DevState &ds)
    {
        auto P = make_params<R>(h, ds);
        k_keys<R, D><<<grid_blocks(h.n, 256, ds.num_sms), 256, 0, ds.stream>>>(P, (const R *)ds.S, ds.sim,
                                                                               ds.keys[0], ds.vals[0]);
    }
    static void permute(const HostParams &h, DevState &ds)
    {
        k_permute<R><<<grid_blocks(h.n, 256, ds.num_sms), 256, 0, ds.stream>>>(
            h.ncomp, h.n, h.npad, (const R *)ds.S, (R *)ds.S2, ds.perm, ds.id, ds.id2, ds.sim, ds.sim2);
    }
    static constexpr bool kReg = (sizeof(R) == 4) || (D == 2);
    static constexpr int kP2GThreads = (D == 3 && kReg) ? 128 : 256;
    static size_t p2g_smem() { return p2g_smem_bytes<R, D, kP2GThreads>(); }
    // one instantiation per material (the staged component count is a compile-time constant)
    template <int MAT> static void p2g_launch(const HostParams &h, DevState &ds)
    {
        auto P = make_params<R>(h, ds);
        if constexpr (sizeof(R) == 4 && MPM_P2G_DIRECT) {
            constexpr int NT = 128;
            constexpr size_t smem = p2g_direct_smem<R, D, NT, MAT>();
            static_assert(smem <= 48 * 1024, "k_p2g_direct shared memory above the default limit");
            // persistent: as many blocks as fit on the GPU at once (3D: the launch
            // bound's MPM_P2G_MINB per SM; 2D: more, its accumulators are 27 values)
            static int per_sm = 0;
            if (per_sm == 0) {
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2g_direct<R, D, NT, MAT>, NT, smem) !=
                        cudaSuccess ||
                    per_sm < 1)
                    per_sm = MPM_P2G_MINB;
            }
            const int nb = ds.num_sms * per_sm;
            // tiles in key order (claiming them largest first, as G2P does, measured slower)
            P2GIO<R> io{(const R *)ds.S, nullptr, h.npad, ds.tiles, ds.counters + 1, ds.counters + 2, ds.posmap,
                        ds.cell_off, (R4<R> *)ds.A, ds.flags};
            k_p2g_direct<R, D, NT, MAT><<<nb, NT, smem, ds.stream>>>(P, io, ds.escaped, ds.counters + 3);
            if (h.transfer == 3) {                   // FLIP: the momenta without forces, for v_i^n
                auto P2 = P;
                P2.no_force = 1;
                P2.save_S = nullptr;
                cudaMemsetAsync(ds.counters + 2, 0, sizeof(int32_t), ds.stream);
                io.A = (R4<R> *)ds.A2;
                k_p2g_direct<R, D, NT, MAT><<<nb, NT, smem, ds.stream>>>(P2, io, ds.escaped, ds.counters + 3);
            }
            return;
        }
        const size_t smem = p2g_smem();
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_p2g<R, D, kReg, kP2GThreads, MAT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
            attr = true;
        }
        int64_t nb = ds.max_tiles;
        const int64_t cap = (int64_t)ds.num_sms * (kP2GThreads == 128 ? MPM_P2G_MINB : 2);
        if (nb > cap) nb = cap;
        if (nb < 1) nb = 1;
        k_p2g<R, D, kReg, kP2GThreads, MAT><<<(int)nb, kP2GThreads, smem, ds.stream>>>(
            P, (const R *)ds.S, ds.tiles, ds.counters, ds.posmap, ds.cell_off, (R4<R> *)ds.A, ds.flags, ds.escaped);
        if (h.transfer == 3) {                       // FLIP: the momenta without forces, for v_i^n
            auto P2 = P;
            P2.no_force = 1;
            P2.save_S = nullptr;
            cudaMemsetAsync(ds.counters + 2, 0, sizeof(int32_t), ds.stream);
            k_p2g<R, D, kReg, kP2GThreads, MAT><<<(int)nb, kP2GThreads, smem, ds.stream>>>(
                P2, (const R *)ds.S, ds.tiles, ds.counters, ds.posmap, ds.cell_off, (R4<R> *)ds.A2, ds.flags,
                ds.escaped);
        }
    }
    static void p2g(const HostParams &h, DevState &ds)
    {
        if (h.material == 1) p2g_launch<1>(h, ds);
        else p2g_launch<0>(h, ds);
    }
    static void grid(const HostParams &h, DevState &ds)
    {
        auto P = make_params<R>(h, ds);
        int64_t nb = h.batch * h.node_tiles_per_sim;        // blocks walk the touched-tile list
        if (nb > (int64_t)ds.num_sms * 8) nb = (int64_t)ds.num_sms * 8;
        k_grid<R, D><<<(unsigned)nb, 256, 0, ds.stream>>>(P, (R4<R> *)ds.A, (R4<R> *)ds.V, ds.flags,
                                                           (R4<R> *)ds.save_A, (R4<R> *)ds.save_V,
                                                           ds.save_L, (R4<R> *)ds.A2, (R4<R> *)ds.V2,
                                                           ds.node_list, ds.counters + 4);
    }
    // the APIC transfer has its own instantiation; the others (TPIC, PIC, FLIP) share one
    template <bool GENERIC, int MAT> static void g2p_launch(const HostParams &h, DevState &ds)
    {
        auto P = make_params<R>(h, ds);
        const size_t smem = G2PSmem<R, D>::total;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_g2p<R, D, GENERIC, MAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
        // persistent: as many blocks as fit at once (3D FP32: the launch bound's two
        // per SM; 2D: three, its registers and shared memory allow it)
        static int per_sm = 0;
        if (per_sm == 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_g2p<R, D, GENERIC, MAT>, G2PSmem<R, D>::NT,
                                                              smem) != cudaSuccess ||
                per_sm < 1)
                per_sm = sizeof(R) == 4 ? MPM_G2P_MINB : 2;
        }
        int64_t nb = ds.max_tiles;
        const int64_t cap = (int64_t)ds.num_sms * per_sm;
        if (nb > cap) nb = cap;
        if (nb < 1) nb = 1;
        k_g2p<R, D, GENERIC, MAT><<<(int)nb, G2PSmem<R, D>::NT, smem, ds.stream>>>(
            P, ds.tmap_V, (R *)ds.S, (const R4<R> *)ds.V, ds.tiles + ds.max_tiles, ds.counters, ds.status,
            (const R4<R> *)ds.V2);
    }
    static void g2p(const HostParams &h, DevState &ds)
    {
        if (h.material == 1) {
            if (h.transfer != 0) g2p_launch<true, 1>(h, ds);
            else g2p_launch<false, 1>(h, ds);
        } else {
            if (h.transfer != 0) g2p_launch<true, 0>(h, ds);
            else g2p_launch<false, 0>(h, ds);
        }
    }
    static void get_field(const HostParams &h, DevState &ds, int field, double *out)
    {
        auto P = make_params<R>(h, ds);
        k_get_field<R, D><<<grid_blocks(h.n, 256, ds.num_sms), 256, 0, ds.stream>>>(P, (const R *)ds.S, ds.id,
                                                                                    field, out);
    }
    static void set_field(const HostParams &h, DevState &ds, int field, const double *in)
    {
        auto P = make_params<R>(h, ds);
        k_set_field<R, D><<<grid_blocks(h.n, 256, ds.num_sms), 256, 0, ds.stream>>>(P, (R *)ds.S, ds.id, field,
                                                                                    in);
    }
    static void diag_particles(const HostParams &h, DevState &ds)
    {
        auto P = make_params<R>(h, ds);
        k_diag_particles<R, D><<<grid_blocks(h.n, 256, ds.num_sms, 4), 256, 0, ds.stream>>>(P, (const R *)ds.S);
    }
};

template <class R> struct Dispatch {
#define MPM_DISPATCH(name, args, call)                       \
    static void name args                                    \
    {                                                        \
        if (h.dim == 2) Launch<R, 2>::call;                  \
        else Launch<R, 3>::call;                             \
    }
    MPM_DISPATCH(init_state, (const HostParams &h, DevState &ds, const double *x, const double *v),
                 init_state(h, ds, x, v))
    MPM_DISPATCH(keys, (const HostParams &h, DevState &ds), keys(h, ds))
    MPM_DISPATCH(permute, (const HostParams &h, DevState &ds), permute(h, ds))
    MPM_DISPATCH(p2g, (const HostParams &h, DevState &ds), p2g(h, ds))
    MPM_DISPATCH(grid, (const HostParams &h, DevState &ds), grid(h, ds))
    MPM_DISPATCH(g2p, (const HostParams &h, DevState &ds), g2p(h, ds))
    MPM_DISPATCH(get_field, (const HostParams &h, DevState &ds, int f, double *o), get_field(h, ds, f, o))
    MPM_DISPATCH(set_field, (const HostParams &h, DevState &ds, int f, const double *i), set_field(h, ds, f, i))
    MPM_DISPATCH(diag_particles, (const HostParams &h, DevState &ds), diag_particles(h, ds))
#undef MPM_DISPATCH
};

}  // namespace mpm
