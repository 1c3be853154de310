// Adjoint (reverse-mode) kernels of the explicit step: the vector-Jacobian
// product of one step S^t -> S^{t+1} (the recursion of Eq. dzda, Sec. 3.1) with
// S = (x, v, C, rho) for the weakly compressible fluid and S = (x, v, C, rho,
// sigma) for Drucker-Prager sand (F and the plastic strain do not feed the
// dynamics and carry no adjoint), and the
// gradient of the tracked-particle loss of Eq. inverse_loss (Sec. 3.2) with
// respect to the wall friction coefficients (Eq. coulomb_friction, Sec. 5.3).
//
// The reverse sweep works on particle states stored in load order (id order),
// independent of the forward pass's sorted order; the grid of each step
// (m, P = q + dt f_int and the post-wall velocity v) is the one the forward
// recompute of the segment saved, so only the reverse kernels run:
//   k_adj_g2p_bwd  adjoint of G2P: scatters v_bar to the grid, x_bar and
//                  rho_bar partials to the particles
//   k_adj_grid_bwd adjoint of the grid update: walls (and d/dmu), division,
//                  over the node tiles the forward step updated
//   k_adj_p2g_bwd  adjoint of P2G: gathers (m_bar, P_bar), completes the
//                  particle adjoint
// Branches (position clamp, wall contact, stick/slide, mass threshold) follow
// the forward pass; the weights' dependence on x_p enters through their
// gradients and Hessians.
#pragma once

#include "mpm_kernels.cuh"

// Resident blocks of 256 threads per SM the reverse particle kernels are compiled for.
#ifndef MPM_ADJ_MINB
#define MPM_ADJ_MINB 2
#endif
// 3D reverse particle kernels in separable (stencil-moment) form, and their
// resident blocks per SM in single precision.
#ifndef MPM_ADJ_SEPARABLE
#define MPM_ADJ_SEPARABLE 1
#endif
#ifndef MPM_ADJ3_MINB
#define MPM_ADJ3_MINB 2
#endif
// Resident blocks per SM of the 3D P2G adjoint in single precision.
#ifndef MPM_ADJ3P_MINB
#define MPM_ADJ3P_MINB 2
#endif

namespace mpm {

// Per-wall device accumulators of dL/dmu (nullptr for walls without friction).
struct MuBar {
    double *w[kMaxWalls];
};

// Second derivatives of the three stencil weights with respect to x.
template <class R> __device__ __forceinline__ void bspline_dd(R inv_dx, R ddw[3])
{
    const R s = inv_dx * inv_dx;
    ddw[0] = s;
    ddw[1] = R(-2) * s;
    ddw[2] = s;
}

// Component count of the adjoint state: (x, v, C, rho), plus the six stress
// components (xx, yy, zz, xy, xz, yz) for Drucker-Prager.
template <int D> __host__ __device__ constexpr int adj_ncomp() { return 2 * D + D * D + 1; }
__host__ __device__ inline int adj_ncomp_material(int dim, int material)
{
    return 2 * dim + dim * dim + 1 + (material == 1 ? 6 : 0);
}

// Reverse of dp_update (Appendix A) for one particle, on the six-component
// stress: given the velocity gradient L (3 x 3, row-major), the stress s before
// the update and the adjoint sb of the updated stress, adds the adjoint of s to
// s_bar and of L to L_bar.  The zone and corner branches of the forward update
// are held fixed.
template <class R>
__device__ __forceinline__ void dp_update_vjp(const Params<R> &P, const R L[9], const R s[6], const R sb[6],
                                              R s_bar[6], R L_bar[9])
{
    const R dt = P.dt;
    const R d0 = dt * L[0], d1 = dt * L[4], d2 = dt * L[8];
    const R d3 = R(0.5) * dt * (L[1] + L[3]);
    const R d4 = R(0.5) * dt * (L[2] + L[6]);
    const R d5 = R(0.5) * dt * (L[5] + L[7]);
    const R w01 = R(0.5) * dt * (L[1] - L[3]);
    const R w02 = R(0.5) * dt * (L[2] - L[6]);
    const R w12 = R(0.5) * dt * (L[5] - L[7]);
    const R S00 = s[0], S11 = s[1], S22 = s[2], S01 = s[3], S02 = s[4], S12 = s[5];
    const R lamK = P.K - R(2) / R(3) * P.G, twoG = R(2) * P.G;
    // forward replay of the trial stress and its invariants
    const R M00 = w01 * S01 + w02 * S02, M11 = -w01 * S01 + w12 * S12, M22 = -w02 * S02 - w12 * S12;
    const R M01 = w01 * S11 + w02 * S12, M10 = -w01 * S00 + w12 * S02;
    const R M02 = w01 * S12 + w02 * S22, M20 = -w02 * S00 - w12 * S01;
    const R M12 = -w01 * S02 + w12 * S22, M21 = -w02 * S01 - w12 * S11;
    const R lt = lamK * (d0 + d1 + d2);
    R t[6];
    t[0] = S00 + R(2) * M00 + lt + twoG * d0;
    t[1] = S11 + R(2) * M11 + lt + twoG * d1;
    t[2] = S22 + R(2) * M22 + lt + twoG * d2;
    t[3] = S01 + M01 + M10 + twoG * d3;
    t[4] = S02 + M02 + M20 + twoG * d4;
    t[5] = S12 + M12 + M21 + twoG * d5;
    const R sm = (t[0] + t[1] + t[2]) / R(3);
    const R dev[6] = {t[0] - sm, t[1] - sm, t[2] - sm, t[3], t[4], t[5]};
    const R tau = rsqrt_(R(0.5) * (dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2]) +
                         dev[3] * dev[3] + dev[4] * dev[4] + dev[5] * dev[5]);
    const R fs = tau - P.k_phi + P.q_phi * sm;
    const R ft = sm - P.sig_t;
    const R h = tau - P.tau_P - P.alpha_P * (sm - P.sig_t);
    // reverse through the return
    R tb[6] = {R(0), R(0), R(0), R(0), R(0), R(0)}, devb[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    R smb = R(0), taub = R(0);
    const R trb = sb[0] + sb[1] + sb[2];
    if (fs <= R(0) && ft < R(0)) {                                   // Zone I: s' = t
#pragma unroll
        for (int k = 0; k < 6; ++k) tb[k] = sb[k];
    } else if ((fs > R(0) && ft < R(0)) || (h > R(0) && ft >= R(0))) {   // Zone II: s' = r dev + smn I
        const R A = P.G + P.K * P.q_phi * P.q_psi;
        const R smn = sm - P.K * P.q_psi * fs / A;
        const bool corner = !P.dp_literal && smn > P.sig_t;
        const R taun = corner ? P.tau_P : P.k_phi - P.q_phi * smn;
        const R r = tau > R(0) ? taun / tau : R(0);
        R rb = R(0);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            rb += sb[k] * dev[k];
            devb[k] = r * sb[k];
        }
        R smnb = corner ? R(0) : trb, taunb = R(0);
        if (tau > R(0)) {
            if (!corner) taunb = rb / tau;
            taub -= rb * taun / (tau * tau);
        }
        smnb -= P.q_phi * taunb;
        smb += smnb * (R(1) - P.K * P.q_psi * P.q_phi / A);
        taub -= smnb * P.K * P.q_psi / A;
    } else {                                                         // Zone III
        const bool corner = !P.dp_literal && tau > P.tau_P;
        if (corner) {                                                // s' = (tau_P / tau) dev + sig_t I
            R rb = R(0);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                rb += sb[k] * dev[k];
                devb[k] = P.tau_P / tau * sb[k];
            }
            taub -= rb * P.tau_P / (tau * tau);
        } else {                                                     // s' = dev + sig_t I
#pragma unroll
            for (int k = 0; k < 6; ++k) devb[k] = sb[k];
        }
    }
    // tau = sqrt(dev_d . dev_d / 2 + dev_o . dev_o)
    if (tau > R(0)) {
#pragma unroll
        for (int k = 0; k < 6; ++k) devb[k] += taub * dev[k] / tau * (k < 3 ? R(0.5) : R(1));
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) tb[k] += devb[k];
    smb -= devb[0] + devb[1] + devb[2];
    tb[0] += smb / R(3);
    tb[1] += smb / R(3);
    tb[2] += smb / R(3);
    // t -> S, M, d
    R Sb[6] = {tb[0], tb[1], tb[2], tb[3], tb[4], tb[5]};
    const R Mb00 = R(2) * tb[0], Mb11 = R(2) * tb[1], Mb22 = R(2) * tb[2];
    const R Mb01 = tb[3], Mb10 = tb[3], Mb02 = tb[4], Mb20 = tb[4], Mb12 = tb[5], Mb21 = tb[5];
    const R ltb = tb[0] + tb[1] + tb[2];
    R db[6] = {twoG * tb[0] + lamK * ltb, twoG * tb[1] + lamK * ltb, twoG * tb[2] + lamK * ltb,
               twoG * tb[3], twoG * tb[4], twoG * tb[5]};
    // M -> S, w   (S index: 0 00, 1 11, 2 22, 3 01, 4 02, 5 12)
    R wb01 = R(0), wb02 = R(0), wb12 = R(0);
    wb01 += Mb00 * S01; Sb[3] += Mb00 * w01; wb02 += Mb00 * S02; Sb[4] += Mb00 * w02;
    wb01 += Mb01 * S11; Sb[1] += Mb01 * w01; wb02 += Mb01 * S12; Sb[5] += Mb01 * w02;
    wb01 += Mb02 * S12; Sb[5] += Mb02 * w01; wb02 += Mb02 * S22; Sb[2] += Mb02 * w02;
    wb01 -= Mb10 * S00; Sb[0] -= Mb10 * w01; wb12 += Mb10 * S02; Sb[4] += Mb10 * w12;
    wb01 -= Mb11 * S01; Sb[3] -= Mb11 * w01; wb12 += Mb11 * S12; Sb[5] += Mb11 * w12;
    wb01 -= Mb12 * S02; Sb[4] -= Mb12 * w01; wb12 += Mb12 * S22; Sb[2] += Mb12 * w12;
    wb02 -= Mb20 * S00; Sb[0] -= Mb20 * w02; wb12 -= Mb20 * S01; Sb[3] -= Mb20 * w12;
    wb02 -= Mb21 * S01; Sb[3] -= Mb21 * w02; wb12 -= Mb21 * S11; Sb[1] -= Mb21 * w12;
    wb02 -= Mb22 * S02; Sb[4] -= Mb22 * w02; wb12 -= Mb22 * S12; Sb[5] -= Mb22 * w12;
#pragma unroll
    for (int k = 0; k < 6; ++k) s_bar[k] += Sb[k];
    // d, w -> L
    const R hdt = R(0.5) * dt;
    L_bar[0] += dt * db[0];
    L_bar[4] += dt * db[1];
    L_bar[8] += dt * db[2];
    L_bar[1] += hdt * (db[3] + wb01);
    L_bar[3] += hdt * (db[3] - wb01);
    L_bar[2] += hdt * (db[4] + wb02);
    L_bar[6] += hdt * (db[4] - wb02);
    L_bar[5] += hdt * (db[5] + wb12);
    L_bar[7] += hdt * (db[5] - wb12);
}

// Walls in order x-, x+, y-, y+, (z-, z+), floor last, applied to u (in place);
// chain[q] receives the input of wall q.
template <class R, int D>
__device__ __forceinline__ void walls_forward(const Params<R> &P, int sim, const int a3[3], R vel[3],
                                              R chain[2 * D][3], bool applied[2 * D])
{
    constexpr int floor_w = 2 * (D - 1);
#pragma unroll
    for (int q = 0; q < 2 * D; ++q) {
        const int w = q < 2 * D - 1 ? (q < floor_w ? q : q + 1) : floor_w;
        const int ax = w >> 1, hi = w & 1;
        const int c = a3[ax] - 2;
        chain[q][0] = vel[0];
        chain[q][1] = vel[1];
        chain[q][2] = vel[2];
        const bool on = hi ? (c >= P.n_cells[ax]) : (c <= 0);
        applied[q] = on;
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
}

// Friction segment index of the node on wall w (as in wall_mu).
template <class R, int D>
__device__ __forceinline__ int64_t wall_seg(const Params<R> &P, int w, const int a3[3])
{
    const WallDev &wd = P.wall[w];
    int s[2] = {0, 0};
#pragma unroll
    for (int q = 0; q < D - 1; ++q) {
        const int ax = wd.seg_axis[q];
        const int c = a3[ax] - 2;
        int sq = c > 0 ? (int)(((int64_t)c * wd.n_seg[q]) / P.n_cells[ax]) : 0;
        s[q] = min(sq, wd.n_seg[q] - 1);
    }
    return (int64_t)s[1] * wd.n_seg[0] + s[0];
}

// Adjoint of the wall chain: ob (adjoint of the output) -> adjoint of u, in place;
// d<ob, out>/d mu is added to mu_bar (per wall segment) for walls with friction.
template <class R, int D>
__device__ __forceinline__ void walls_backward(const Params<R> &P, int sim, const int a3[3],
                                               const R chain[2 * D][3], const bool applied[2 * D], R ob[3],
                                               double *const mu_bar[kMaxWalls])
{
    constexpr int floor_w = 2 * (D - 1);
#pragma unroll
    for (int q = 2 * D - 1; q >= 0; --q) {
        if (!applied[q]) continue;
        const int w = q < 2 * D - 1 ? (q < floor_w ? q : q + 1) : floor_w;
        const int ax = w >> 1, hi = w & 1;
        const R *u = chain[q];
        const R sgn = hi ? R(1) : R(-1);
        const R vn = sgn * u[ax];
        if (!(vn > R(0))) continue;                  // contact not active: identity
        const R mu = wall_mu<R, D>(P, w, sim, a3);
        if (!(mu > R(0))) {                          // slip: normal component removed
            ob[ax] = R(0);
            continue;
        }
        R vt2 = R(0);
#pragma unroll
        for (int bb = 0; bb < D; ++bb)
            if (bb != ax) vt2 += u[bb] * u[bb];
        const R vt = rsqrt_(vt2);
        if (vt <= mu * vn) {                         // stick: output 0
            ob[0] = ob[1] = ob[2] = R(0);
            continue;
        }
        const R s = R(1) - mu * vn / vt;
        R dot = R(0);
#pragma unroll
        for (int bb = 0; bb < D; ++bb)
            if (bb != ax) dot += ob[bb] * u[bb];
        const R k = dot * mu * vn / (vt * vt * vt);
#pragma unroll
        for (int bb = 0; bb < D; ++bb)
            if (bb != ax) ob[bb] = s * ob[bb] + k * u[bb];
        ob[ax] = -dot * mu * sgn / vt;
        if (mu_bar[w] != nullptr)
            atomicAdd(&mu_bar[w][(int64_t)sim * P.wall[w].n_seg[0] * P.wall[w].n_seg[1] + wall_seg<R, D>(P, w, a3)],
                      (double)(-dot * vn / vt));
    }
}

// State component of adjoint component c < 2D + D^2 (the adjoint order is x, v, C, rho [, sigma]).
template <int D, class R> __device__ __forceinline__ int adj_state_comp(const Params<R> &P, int c)
{
    return c < D ? P.off_x + c : (c < 2 * D ? P.off_v + (c - D) : P.off_C + (c - 2 * D));
}

// Particle state gather (slot order -> load order) and scatter.
template <class R, int D>
__global__ void k_adj_save(const Params<R> P, const R *__restrict__ S, const int32_t *__restrict__ id,
                           R *__restrict__ dst)
{
    constexpr int NA = adj_ncomp<D>();
    const int nsig = P.material == 1 ? 6 : 0;
    const int64_t n = P.n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = id[i];
        const R *Sp = S + sblock(i, P.ncomp);
#pragma unroll
        for (int c = 0; c < NA - 1; ++c) dst[c * n + o] = Sp[adj_state_comp<D>(P, c) * kPB];
        dst[(NA - 1) * n + o] = Sp[P.off_rho * kPB];
        for (int k = 0; k < nsig; ++k) dst[(NA + k) * n + o] = Sp[(P.off_sig + k) * kPB];
    }
}

template <class R, int D>
__global__ void k_adj_restore(const Params<R> P, R *__restrict__ S, const int32_t *__restrict__ id,
                              const R *__restrict__ src)
{
    constexpr int NA = adj_ncomp<D>();
    const int nsig = P.material == 1 ? 6 : 0;
    const int64_t n = P.n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = id[i];
        R *Sp = S + sblock(i, P.ncomp);
#pragma unroll
        for (int c = 0; c < NA - 1; ++c) Sp[adj_state_comp<D>(P, c) * kPB] = src[c * n + o];
        Sp[P.off_rho * kPB] = src[(NA - 1) * n + o];
        for (int k = 0; k < nsig; ++k) Sp[(P.off_sig + k) * kPB] = src[(NA + k) * n + o];
    }
}

// Positions of the tracked particles (load-order ids) -> out[track].
template <class R, int D>
__global__ void k_adj_track(const Params<R> P, const R *__restrict__ S, const int32_t *__restrict__ id,
                            const int32_t *__restrict__ track_of_id, double *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int l = track_of_id[id[i]];
        if (l < 0) continue;
#pragma unroll
        for (int a = 0; a < D; ++a) out[(int64_t)l * D + a] = (double)S[sblock(i, P.ncomp) + (P.off_x + a) * kPB];
    }
}

// lam.x[id_l] += 2 (x_l - z_l) for the tracked particles of one observation.
template <class R, int D>
__global__ void k_adj_seed(int64_t n, int n_track, const int64_t *__restrict__ ids, const double *__restrict__ x_obs,
                           const double *__restrict__ z_obs, R *__restrict__ lam)
{
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n_track; l += gridDim.x * blockDim.x) {
        const int64_t o = ids[l];
#pragma unroll
        for (int a = 0; a < D; ++a)
            atomicAdd(&lam[a * n + o], (R)(2.0 * (x_obs[(int64_t)l * D + a] - z_obs[(int64_t)l * D + a])));
    }
}

// pos[id[slot]] = slot.
template <class R>
__global__ void k_adj_inverse(int64_t n, const int32_t *__restrict__ id, int32_t *__restrict__ pos)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pos[id[i]] = (int32_t)i;
}

// Re-order an adjoint state from the order with inverse map pos_old to the
// order with ids id_new: out[c n + s] = in[c n + pos_old[id_new[s]]].
template <class R>
__global__ void k_adj_reorder(int64_t n, int nc, const int32_t *__restrict__ pos_old,
                              const int32_t *__restrict__ id_new, const R *__restrict__ in, R *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t src = pos_old[id_new[i]];
        for (int c = 0; c < nc; ++c) out[c * n + i] = in[c * n + src];
    }
}

// lam.x[slot] += 2 (x_l - z_l) for the tracked particles (slot order with ids id).
template <class R, int D>
__global__ void k_adj_seed_slots(int64_t n, const int32_t *__restrict__ id, const int32_t *__restrict__ track_of_id,
                                 const double *__restrict__ x_obs, const double *__restrict__ z_obs,
                                 R *__restrict__ lam)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int l = track_of_id[id[i]];
        if (l < 0) continue;
#pragma unroll
        for (int a = 0; a < D; ++a)
            lam[a * n + i] += (R)(2.0 * (x_obs[(int64_t)l * D + a] - z_obs[(int64_t)l * D + a]));
    }
}

// Velocity monitors (Sec. 5.2, Case 3: the mean velocity of the particles inside
// each monitor region).  Per closed box [lo, hi] (boxes: n_mon x 2 x D doubles,
// low corner then high corner) the sum of v_p and the count of the particles
// with x_p inside: sums[l (D + 1) + a] (a < D) and sums[l (D + 1) + D].  x and v
// point at the first component of a state view (sview: component-major with
// stride ld > 0, or the blocked particle state with -ld components).  Block sums in shared memory, then one
// FP64 atomic per monitor and value.
template <class R, int D>
__global__ void __launch_bounds__(256) k_monitor_sum(int64_t n, int64_t ld, const R *__restrict__ x,
                                                     const R *__restrict__ v, int n_mon,
                                                     const double *__restrict__ boxes, double *__restrict__ sums)
{
    __shared__ double acc[kMaxMonitors * (D + 1)];
    for (int i = threadIdx.x; i < n_mon * (D + 1); i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double xp[D];
#pragma unroll
        for (int a = 0; a < D; ++a) xp[a] = (double)sview(x, ld, a, i);
        for (int l = 0; l < n_mon; ++l) {
            const double *b = boxes + (int64_t)l * 2 * D;
            bool in = true;
#pragma unroll
            for (int a = 0; a < D; ++a) in = in && xp[a] >= b[a] && xp[a] <= b[D + a];
            if (!in) continue;
#pragma unroll
            for (int a = 0; a < D; ++a) atomicAdd(&acc[l * (D + 1) + a], (double)sview(v, ld, a, i));
            atomicAdd(&acc[l * (D + 1) + D], 1.0);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_mon * (D + 1); i += blockDim.x)
        if (acc[i] != 0.0) atomicAdd(&sums[i], acc[i]);
}

// Adjoint seed of the monitor loss sum_l |Q_l - z_l|^2: for every particle inside
// monitor l, lam.v += g_l with g_l = 2 (Q_l - z_l) / |P_l| (membership held fixed).
// x: the first position component of a state view (sview), in the order of lam.
template <class R, int D>
__global__ void k_monitor_seed(int64_t n, int64_t ld, const R *__restrict__ x, int n_mon,
                               const double *__restrict__ boxes, const double *__restrict__ g, R *__restrict__ lam)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double xp[D];
#pragma unroll
        for (int a = 0; a < D; ++a) xp[a] = (double)sview(x, ld, a, i);
        for (int l = 0; l < n_mon; ++l) {
            const double *b = boxes + (int64_t)l * 2 * D;
            bool in = true;
#pragma unroll
            for (int a = 0; a < D; ++a) in = in && xp[a] >= b[a] && xp[a] <= b[D + a];
            if (!in) continue;
#pragma unroll
            for (int a = 0; a < D; ++a) lam[(D + a) * n + i] += (R)g[l * D + a];
        }
    }
}

// Load-order copy of w components of an adjoint state: out[id[s] w + k] = lam[(off + k) n + s].
template <class R>
__global__ void k_adj_gather(int64_t n, int w, int off, const int32_t *__restrict__ id, const R *__restrict__ lam,
                             double *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < w; ++k) out[(int64_t)id[i] * w + k] = (double)lam[(int64_t)(off + k) * n + i];
}

// The inverse: an adjoint state from a load-order array, lam[(off + k) n + s] = in[id[s] w + k].
template <class R>
__global__ void k_adj_scatter_in(int64_t n, int w, int off, const int32_t *__restrict__ id,
                                 const double *__restrict__ in, R *__restrict__ lam)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < w; ++k) lam[(int64_t)(off + k) * n + i] = (R)in[(int64_t)id[i] * w + k];
}

template <class R>
__global__ void k_adj_zero(R *__restrict__ p, int64_t count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = R(0);
}

// Stencil data of one particle for the reverse kernels.
template <class R, int D> struct AdjStencil {
    int b[D];
    R fx[D], w[D][3], dw[D][3], ddw[3];
};

template <class R, int D>
__device__ __forceinline__ void adj_stencil(const Params<R> &P, const R x[D], AdjStencil<R, D> &s)
{
#pragma unroll
    for (int a = 0; a < D; ++a) {
        s.b[a] = base_cell(x[a], P.inv_dx, P.n_cells[a]);
        s.fx[a] = x[a] * P.inv_dx - R(s.b[a]);
        bspline(s.fx[a], P.inv_dx, s.w[a], s.dw[a]);
    }
    bspline_dd(P.inv_dx, s.ddw);
}

// Weight, gradient and Hessian of stencil node (k0, k1, k2).
template <class R, int D>
__device__ __forceinline__ void adj_node(const AdjStencil<R, D> &s, const int kk[3], R &w, R g[D], R H[D][D])
{
    R f[D], df[D], ddf[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        f[a] = s.w[a][kk[a]];
        df[a] = s.dw[a][kk[a]];
        ddf[a] = s.ddw[kk[a]];
    }
    w = R(1);
#pragma unroll
    for (int a = 0; a < D; ++a) w *= f[a];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        R ga = df[a];
#pragma unroll
        for (int c = 0; c < D; ++c)
            if (c != a) ga *= f[c];
        g[a] = ga;
#pragma unroll
        for (int b = 0; b < D; ++b) {
            R h = R(1);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const int cnt = (c == a) + (c == b);
                h *= cnt == 0 ? f[c] : (cnt == 1 ? df[c] : ddf[c]);
            }
            H[a][b] = h;
        }
    }
}

// Adjoint of G2P for one particle: lam_in is the adjoint of S^{t+1}; writes the
// G2P part of the adjoint of x and rho to lam_out and scatters v_bar to GVB.
template <class R, int D>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? MPM_ADJ_MINB : 1) k_adj_g2p_bwd(const Params<R> P, const R *__restrict__ st, const R4<R> *__restrict__ GV,
                              const R *__restrict__ lam_in, R *__restrict__ lam_out, R4<R> *__restrict__ GVB)
{
    const int64_t n = P.n;
    constexpr int JC = 2 * D, JR = 2 * D + D * D;
    const R cscale = R(4) * P.inv_dx;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        R x[D];
#pragma unroll
        for (int a = 0; a < D; ++a) x[a] = st[a * n + p];
        AdjStencil<R, D> s;
        adj_stencil<R, D>(P, x, s);
        // forward quantities: v_p and L
        R vp[D], Lf[D * D];
#pragma unroll
        for (int a = 0; a < D; ++a) vp[a] = R(0);
#pragma unroll
        for (int q = 0; q < D * D; ++q) Lf[q] = R(0);
#pragma unroll
        for (int k = 0; k < Geo<D>::STENCIL; ++k) {
            const int kk[3] = {k % 3, (k / 3) % 3, k / 9};
            R w, g[D], H[D][D];
            adj_node<R, D>(s, kk, w, g, H);
            int a3[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < D; ++a) a3[a] = s.b[a] + 2 + kk[a];
            const R4<R> v4 = GV[lin3<D>(a3, P.G_nodes)];
            const R vi[3] = {v4.x, v4.y, v4.z};
#pragma unroll
            for (int a = 0; a < D; ++a) {
                vp[a] += w * vi[a];
#pragma unroll
                for (int b = 0; b < D; ++b) Lf[a * D + b] += vi[a] * g[b];
            }
        }
        R trL = R(0);
#pragma unroll
        for (int a = 0; a < D; ++a) trL += Lf[a * D + a];
        // adjoints of the outputs
        R xb[D], vbt[D], Cb[D * D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const R xo = lam_in[a * n + p];
            const R xn = x[a] + P.dt * vp[a];
            const bool clamped = xn < R(0) || xn > P.L[a];
            xb[a] = clamped ? R(0) : xo;
            vbt[a] = lam_in[(D + a) * n + p] + (clamped ? R(0) : P.dt * xo);
        }
#pragma unroll
        for (int q = 0; q < D * D; ++q) Cb[q] = lam_in[(JC + q) * n + p];
        const R rho = st[JR * n + p];
        const R den = R(1) + P.dt * trL;
        const R rb1 = lam_in[JR * n + p];
        const R rhob = rb1 / den;
        const R trLb = -rb1 * rho * P.dt / (den * den);
        // adjoint of L: the density path, and for Drucker-Prager the stress update
        R Lb[D * D];
#pragma unroll
        for (int q = 0; q < D * D; ++q) Lb[q] = R(0);
#pragma unroll
        for (int a = 0; a < D; ++a) Lb[a * D + a] = trLb;
        if (P.material == 1) {
            R L3[9], Lb3[9], s6[6], sb6[6], s0b[6];
#pragma unroll
            for (int q = 0; q < 9; ++q) L3[q] = Lb3[q] = R(0);
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = 0; b < D; ++b) L3[a * 3 + b] = Lf[a * D + b];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                s6[k] = st[(JR + 1 + k) * n + p];
                sb6[k] = lam_in[(JR + 1 + k) * n + p];
                s0b[k] = R(0);
            }
            dp_update_vjp<R>(P, L3, s6, sb6, s0b, Lb3);
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = 0; b < D; ++b) Lb[a * D + b] += Lb3[a * 3 + b];
#pragma unroll
            for (int k = 0; k < 6; ++k) lam_out[(JR + 1 + k) * n + p] = s0b[k];
        }
        // x_bar through (k - fx): C = (4 / dx) sum w v (k - fx) and dfx/dx = 1/dx
#pragma unroll
        for (int b = 0; b < D; ++b) {
            R sacc = R(0);
#pragma unroll
            for (int a = 0; a < D; ++a) sacc += Cb[a * D + b] * vp[a];
            xb[b] -= cscale * P.inv_dx * sacc;
        }
#pragma unroll
        for (int k = 0; k < Geo<D>::STENCIL; ++k) {
            const int kk[3] = {k % 3, (k / 3) % 3, k / 9};
            R w, g[D], H[D][D];
            adj_node<R, D>(s, kk, w, g, H);
            int a3[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < D; ++a) a3[a] = s.b[a] + 2 + kk[a];
            const int64_t gi = lin3<D>(a3, P.G_nodes);
            const R4<R> v4 = GV[gi];
            const R vi[3] = {v4.x, v4.y, v4.z};
            R vb[3] = {R(0), R(0), R(0)};
            R wbar = R(0), gbar[D];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                R cr = R(0);
#pragma unroll
                for (int b = 0; b < D; ++b) cr += Cb[a * D + b] * (R(kk[b]) - s.fx[b]);
                R Lg = R(0);
#pragma unroll
                for (int b = 0; b < D; ++b) Lg += Lb[a * D + b] * g[b];
                vb[a] = w * vbt[a] + cscale * w * cr + Lg;
                wbar += vbt[a] * vi[a] + cscale * cr * vi[a];
            }
#pragma unroll
            for (int b = 0; b < D; ++b) {
                R gb = R(0);
#pragma unroll
                for (int a = 0; a < D; ++a) gb += Lb[a * D + b] * vi[a];
                gbar[b] = gb;
            }
#pragma unroll
            for (int b = 0; b < D; ++b) {
                R hb = R(0);
#pragma unroll
                for (int a = 0; a < D; ++a) hb += H[b][a] * gbar[a];
                xb[b] += wbar * g[b] + hb;
            }
            red_add4(&GVB[gi], vb[0], vb[1], vb[2], R(0));
        }
#pragma unroll
        for (int a = 0; a < D; ++a) lam_out[a * n + p] = xb[a];
        lam_out[JR * n + p] = rhob;
    }
}

// Adjoint of the grid update per node: GVB (adjoint of v) -> GAB (adjoint of m, P)
// over the node tiles the forward step updated (the list GL it saved: GL[0] tiles,
// then their indices), blocks striding the list; GVB is cleared behind, ready for
// the next reverse step.
template <class R, int D>
__global__ void __launch_bounds__(256) k_adj_grid_bwd(const Params<R> P, const R4<R> *__restrict__ GA,
                                                      R4<R> *__restrict__ GVB, R4<R> *__restrict__ GAB,
                                                      const int32_t *__restrict__ GL, MuBar mu_bar,
                                                      int32_t *__restrict__ scatter_cursor)
{
    using Gm = Geo<D>;
    if (scatter_cursor != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *scatter_cursor = 0;
    const int n_list = GL[0];
    for (int li = blockIdx.x; li < n_list; li += gridDim.x) {
    const int64_t ut = GL[1 + li];
    int u[3] = {0, 0, 0};
    int64_t r = ut;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        u[a] = (int)(r % P.node_tiles[a]);
        r /= P.node_tiles[a];
    }
    for (int t = threadIdx.x; t < Gm::TN; t += blockDim.x) {
        int a3[3] = {0, 0, 0};
        int rr = t;
        bool ok = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            a3[a] = u[a] * Gm::T + rr % Gm::T;
            rr /= Gm::T;
            ok = ok && a3[a] < P.G_nodes[a];
        }
        if (!ok) continue;
        const int64_t i = lin3<D>(a3, P.G_nodes);
        const R4<R> b4 = GVB[i];
        GVB[i] = R4<R>{R(0), R(0), R(0), R(0)};
        const R4<R> acc = GA[i];
        if (!(acc.x > P.m_eps)) {
            GAB[i] = R4<R>{R(0), R(0), R(0), R(0)};
            continue;
        }
        const R inv_m = R(1) / acc.x;
        R vel[3] = {acc.y * inv_m + P.dt * P.gravity[0], acc.z * inv_m + P.dt * P.gravity[1],
                    D == 3 ? acc.w * inv_m + P.dt * P.gravity[2] : R(0)};
        R chain[2 * D][3];
        bool applied[2 * D];
        const unsigned removed = obstacle_contact<R, D>(P, a3, vel);
        walls_forward<R, D>(P, 0, a3, vel, chain, applied);
        R ob[3] = {b4.x, b4.y, b4.z};
        walls_backward<R, D>(P, 0, a3, chain, applied, ob, mu_bar.w);
#pragma unroll
        for (int a = 0; a < D; ++a)                  // the obstacle projections (their own transposes)
            if ((removed >> a) & 1u) ob[a] = R(0);
        const R Pv[3] = {acc.y, acc.z, acc.w};
        R mb = R(0);
#pragma unroll
        for (int a = 0; a < D; ++a) mb -= ob[a] * Pv[a] * inv_m * inv_m;
        GAB[i] = R4<R>{mb, ob[0] * inv_m, ob[1] * inv_m, D == 3 ? ob[2] * inv_m : R(0)};
    }
    }
}

// Adjoint of P2G for one particle; completes lam_out (adjoint of S^t).
template <class R, int D>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? MPM_ADJ_MINB : 1) k_adj_p2g_bwd(const Params<R> P, const R *__restrict__ st, const R4<R> *__restrict__ GAB,
                              R *__restrict__ lam_out)
{
    const int64_t n = P.n;
    constexpr int JV = D, JC = 2 * D, JR = 2 * D + D * D;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        R x[D], v[D], C[D * D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            x[a] = st[a * n + p];
            v[a] = st[(JV + a) * n + p];
        }
#pragma unroll
        for (int q = 0; q < D * D; ++q) C[q] = st[(JC + q) * n + p];
        const R rho = st[JR * n + p];
        const R mp = P.mass;
        const bool sand = P.material == 1;
        const R pr = sand ? R(0) : tait(P, rho);
        const R sforce = P.dt * mp / rho * pr;             // fluid: P += sforce * grad w  (sigma = -p I)
        // Drucker-Prager: P_a += Fm_ab grad_b w with Fm = -dt (m / rho) sigma
        R Fm[D * D], Fmb[D * D];
        if (sand) {
            R s6[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) s6[k] = st[(JR + 1 + k) * n + p];
            const R c = -P.dt * mp / rho;
            const int ix[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = 0; b < D; ++b) Fm[a * D + b] = c * s6[ix[a][b]];
        }
#pragma unroll
        for (int q = 0; q < D * D; ++q) Fmb[q] = R(0);
        AdjStencil<R, D> s;
        adj_stencil<R, D>(P, x, s);
        R xb[D], vb[D], Cb[D * D], sb = R(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            xb[a] = R(0);
            vb[a] = R(0);
        }
#pragma unroll
        for (int q = 0; q < D * D; ++q) Cb[q] = R(0);
#pragma unroll
        for (int k = 0; k < Geo<D>::STENCIL; ++k) {
            const int kk[3] = {k % 3, (k / 3) % 3, k / 9};
            R w, g[D], H[D][D];
            adj_node<R, D>(s, kk, w, g, H);
            int a3[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < D; ++a) a3[a] = s.b[a] + 2 + kk[a];
            const R4<R> ab = GAB[lin3<D>(a3, P.G_nodes)];
            const R Pb[3] = {ab.y, ab.z, ab.w};
            R rr[D];
#pragma unroll
            for (int b = 0; b < D; ++b) rr[b] = (R(kk[b]) - s.fx[b]) * P.dx;
            R wbar = mp * ab.x, gbar[D];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                R aff = v[a];
#pragma unroll
                for (int b = 0; b < D; ++b) aff += C[a * D + b] * rr[b];
                wbar += mp * Pb[a] * aff;
                vb[a] += mp * w * Pb[a];
#pragma unroll
                for (int b = 0; b < D; ++b) {
                    Cb[a * D + b] += mp * w * Pb[a] * rr[b];
                    xb[b] -= mp * w * Pb[a] * C[a * D + b];
                }
                if (sand) {
#pragma unroll
                    for (int b = 0; b < D; ++b) Fmb[a * D + b] += Pb[a] * g[b];
                } else {
                    gbar[a] = sforce * Pb[a];
                    sb += Pb[a] * g[a];
                }
            }
            if (sand) {
#pragma unroll
                for (int b = 0; b < D; ++b) {
                    R gb = R(0);
#pragma unroll
                    for (int a = 0; a < D; ++a) gb += Fm[a * D + b] * Pb[a];
                    gbar[b] = gb;
                }
            }
#pragma unroll
            for (int b = 0; b < D; ++b) {
                R hb = R(0);
#pragma unroll
                for (int a = 0; a < D; ++a) hb += H[b][a] * gbar[a];
                xb[b] += wbar * g[b] + hb;
            }
        }
        if (sand) {
            // Fm = -dt (m / rho) sigma: adjoints of the six stress components and of rho
            const R c = -P.dt * mp / rho;
            R s6b[6] = {R(0), R(0), R(0), R(0), R(0), R(0)}, rhob = R(0);
            const int ix[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = 0; b < D; ++b) {
                    s6b[ix[a][b]] += c * Fmb[a * D + b];
                    rhob -= Fmb[a * D + b] * Fm[a * D + b] / rho;
                }
#pragma unroll
            for (int a = 0; a < D; ++a) {
                lam_out[a * n + p] += xb[a];
                lam_out[(JV + a) * n + p] = vb[a];
            }
#pragma unroll
            for (int q = 0; q < D * D; ++q) lam_out[(JC + q) * n + p] = Cb[q];
            lam_out[JR * n + p] += rhob;
#pragma unroll
            for (int k = 0; k < 6; ++k) lam_out[(JR + 1 + k) * n + p] += s6b[k];
            continue;
        }
        // sforce = dt m p(rho) / rho
        const R r1 = rho * P.inv_rho0;
        R dp = P.bulk_K * P.inv_rho0;                      // dp/drho = (K / rho0) (rho / rho0)^(gamma - 1)
        if (P.gamma_int > 0) {
            for (int k = 1; k < P.gamma_int; ++k) dp *= r1;
        } else {
            dp *= pow(r1, P.gamma - R(1));
        }
        const R dsdrho = P.dt * mp * (dp * rho - pr) / (rho * rho);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            lam_out[a * n + p] += xb[a];
            lam_out[(JV + a) * n + p] = vb[a];
        }
#pragma unroll
        for (int q = 0; q < D * D; ++q) lam_out[(JC + q) * n + p] = Cb[q];
        lam_out[JR * n + p] += sb * dsdrho;
    }
}

// ------------------------------------------------------------------ 3D reverse kernels in separable form

// Stencil moments of a three-component node field f (and optionally the L
// moments of a scalar node field g) in 3D, contracted one axis at a time.  With
// node offsets k_a in {0, 1, 2}, weight w = w_0 w_1 w_2 and d_b w its b-derivative:
//   V       = sum w f            M[b]    = sum k_b w f       L[b] = sum d_b w f
//   Q[c][b] = sum k_c d_b w f    H[p]    = sum d_b d_a w f   (p: 00, 11, 22, 01, 02, 12)
//   Lg[b]   = sum d_b w g
// (all [..][comp]).  Per axis the factors are w, dw, k w, k dw and the constant
// second derivative of the quadratic B-spline.
template <class R> struct Mom3 {
    R V[3], M[3][3], L[3][3], Q[3][3][3], H[6][3], Lg[3];
};

template <class R, bool WITH_G, class Load>
__device__ __forceinline__ void stencil_moments3(const R w[3][3], const R dw[3][3], R inv_dx, Load load, Mom3<R> &m)
{
    const R s2 = inv_dx * inv_dx;
    const R dd[3] = {s2, R(-2) * s2, s2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        m.V[c] = m.Lg[c] = R(0);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            m.M[b][c] = m.L[b][c] = R(0);
#pragma unroll
            for (int e = 0; e < 3; ++e) m.Q[e][b][c] = R(0);
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) m.H[q][c] = R(0);
    }
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2) {
        // the slice's nine node values are loaded up front (their latencies overlap)
        R fs[9][3], gs[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) load(q % 3, q / 3, k2, fs[q], gs[q]);
        // prefixes over axes 0 and 1 (first letter axis 0, second axis 1)
        R WW[3], DW[3], WD[3], JW[3], WJ[3], JDW[3], WJD[3], JD[3], DJ[3], DDW[3], WDD[3], DDp[3];
        R gWW = R(0), gDW = R(0), gWD = R(0);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            WW[c] = DW[c] = WD[c] = JW[c] = WJ[c] = JDW[c] = WJD[c] = JD[c] = DJ[c] = DDW[c] = WDD[c] = DDp[c] = R(0);
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            R XW[3], XD[3], XJ[3], XJD[3], XDD[3];
            R gW = R(0), gD = R(0);
#pragma unroll
            for (int c = 0; c < 3; ++c) XW[c] = XD[c] = XJ[c] = XJD[c] = XDD[c] = R(0);
#pragma unroll
            for (int k0 = 0; k0 < 3; ++k0) {
                const R *f = fs[k1 * 3 + k0];
                const R g = gs[k1 * 3 + k0];
                const R a0 = w[0][k0], b0 = dw[0][k0];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    XW[c] += a0 * f[c];
                    XD[c] += b0 * f[c];
                    if (k0 > 0) {
                        XJ[c] += R(k0) * a0 * f[c];
                        XJD[c] += R(k0) * b0 * f[c];
                    }
                    XDD[c] += dd[k0] * f[c];
                }
                if (WITH_G) {
                    gW += a0 * g;
                    gD += b0 * g;
                }
            }
            const R a1 = w[1][k1], b1 = dw[1][k1], j1 = R(k1) * a1, jd1 = R(k1) * b1, c1 = dd[k1];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                WW[c] += a1 * XW[c];
                DW[c] += a1 * XD[c];
                WD[c] += b1 * XW[c];
                JW[c] += a1 * XJ[c];
                WJ[c] += j1 * XW[c];
                JDW[c] += a1 * XJD[c];
                WJD[c] += jd1 * XW[c];
                JD[c] += b1 * XJ[c];
                DJ[c] += j1 * XD[c];
                DDW[c] += a1 * XDD[c];
                WDD[c] += c1 * XW[c];
                DDp[c] += b1 * XD[c];
            }
            if (WITH_G) {
                gWW += a1 * gW;
                gDW += a1 * gD;
                gWD += b1 * gW;
            }
        }
        const R a2 = w[2][k2], b2 = dw[2][k2], j2 = R(k2) * a2, jd2 = R(k2) * b2, c2 = dd[k2];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            m.V[c] += a2 * WW[c];
            m.M[0][c] += a2 * JW[c];
            m.M[1][c] += a2 * WJ[c];
            m.M[2][c] += j2 * WW[c];
            m.L[0][c] += a2 * DW[c];
            m.L[1][c] += a2 * WD[c];
            m.L[2][c] += b2 * WW[c];
            m.Q[0][0][c] += a2 * JDW[c];
            m.Q[1][1][c] += a2 * WJD[c];
            m.Q[2][2][c] += jd2 * WW[c];
            m.Q[0][1][c] += a2 * JD[c];
            m.Q[0][2][c] += b2 * JW[c];
            m.Q[1][0][c] += a2 * DJ[c];
            m.Q[1][2][c] += b2 * WJ[c];
            m.Q[2][0][c] += j2 * DW[c];
            m.Q[2][1][c] += j2 * WD[c];
            m.H[0][c] += a2 * DDW[c];
            m.H[1][c] += a2 * WDD[c];
            m.H[2][c] += c2 * WW[c];
            m.H[3][c] += a2 * DDp[c];
            m.H[4][c] += b2 * DW[c];
            m.H[5][c] += b2 * WD[c];
        }
        if (WITH_G) {
            m.Lg[0] += a2 * gDW;
            m.Lg[1] += a2 * gWD;
            m.Lg[2] += b2 * gWW;
        }
    }
}

// The same moments in single precision with paired arithmetic: components PC
// and PC + 1 of the node field run as one paired fused multiply-add (__ffma2_rn,
// each half rounded as fmaf) against a factor broadcast into both halves, the
// third component stays scalar; the sums are bitwise those of the form above.
// PC is chosen so that the paired components are an aligned pair of the node's
// 16-byte load.
template <int PC, bool WITH_G, class Load>
__device__ __forceinline__ void stencil_moments3_x2(const float w[3][3], const float dw[3][3], float inv_dx, Load load,
                                                    Mom3<float> &m)
{
    constexpr int SC = PC == 0 ? 2 : 0;             // the scalar component
    auto bc = [](float a) { return make_float2(a, a); };
    auto z2 = []() { return make_float2(0.f, 0.f); };
    const float s2 = inv_dx * inv_dx;
    const float dd[3] = {s2, -2.f * s2, s2};
    float2 V = z2(), M[3], L[3], Q[3][3], H[6];
    float v_ = 0.f, M_[3], L_[3], Q_[3][3], H_[6], Lg[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        M[b] = L[b] = z2();
        M_[b] = L_[b] = 0.f;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            Q[e][b] = z2();
            Q_[e][b] = 0.f;
        }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        H[q] = z2();
        H_[q] = 0.f;
    }
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2) {
        float2 fp[9];
        float fsc[9], gs[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            float f[3], g;
            load(q % 3, q / 3, k2, f, g);
            fp[q] = make_float2(f[PC], f[PC + 1]);
            fsc[q] = f[SC];
            gs[q] = g;
        }
        float2 WW = z2(), DW = z2(), WD = z2(), JW = z2(), WJ = z2(), JDW = z2(), WJD = z2(), JD = z2(), DJ = z2(),
               DDW = z2(), WDD = z2(), DDp = z2();
        float ww = 0.f, dw_ = 0.f, wd = 0.f, jw = 0.f, wj = 0.f, jdw = 0.f, wjd = 0.f, jd = 0.f, dj = 0.f, ddw = 0.f,
              wdd = 0.f, ddp = 0.f;
        float gWW = 0.f, gDW = 0.f, gWD = 0.f;
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            float2 XW = z2(), XD = z2(), XJ = z2(), XJD = z2(), XDD = z2();
            float xw = 0.f, xd = 0.f, xj = 0.f, xjd = 0.f, xdd = 0.f, gW = 0.f, gD = 0.f;
#pragma unroll
            for (int k0 = 0; k0 < 3; ++k0) {
                const float2 f = fp[k1 * 3 + k0];
                const float fs = fsc[k1 * 3 + k0];
                const float a0 = w[0][k0], b0 = dw[0][k0];
                XW = __ffma2_rn(bc(a0), f, XW);
                xw = fmaf(a0, fs, xw);
                XD = __ffma2_rn(bc(b0), f, XD);
                xd = fmaf(b0, fs, xd);
                if (k0 > 0) {
                    XJ = __ffma2_rn(bc(float(k0) * a0), f, XJ);
                    xj = fmaf(float(k0) * a0, fs, xj);
                    XJD = __ffma2_rn(bc(float(k0) * b0), f, XJD);
                    xjd = fmaf(float(k0) * b0, fs, xjd);
                }
                XDD = __ffma2_rn(bc(dd[k0]), f, XDD);
                xdd = fmaf(dd[k0], fs, xdd);
                if (WITH_G) {
                    gW = fmaf(a0, gs[k1 * 3 + k0], gW);
                    gD = fmaf(b0, gs[k1 * 3 + k0], gD);
                }
            }
            const float a1 = w[1][k1], b1 = dw[1][k1], j1 = float(k1) * a1, jd1 = float(k1) * b1, c1 = dd[k1];
            WW = __ffma2_rn(bc(a1), XW, WW);     ww = fmaf(a1, xw, ww);
            DW = __ffma2_rn(bc(a1), XD, DW);     dw_ = fmaf(a1, xd, dw_);
            WD = __ffma2_rn(bc(b1), XW, WD);     wd = fmaf(b1, xw, wd);
            JW = __ffma2_rn(bc(a1), XJ, JW);     jw = fmaf(a1, xj, jw);
            WJ = __ffma2_rn(bc(j1), XW, WJ);     wj = fmaf(j1, xw, wj);
            JDW = __ffma2_rn(bc(a1), XJD, JDW);  jdw = fmaf(a1, xjd, jdw);
            WJD = __ffma2_rn(bc(jd1), XW, WJD);  wjd = fmaf(jd1, xw, wjd);
            JD = __ffma2_rn(bc(b1), XJ, JD);     jd = fmaf(b1, xj, jd);
            DJ = __ffma2_rn(bc(j1), XD, DJ);     dj = fmaf(j1, xd, dj);
            DDW = __ffma2_rn(bc(a1), XDD, DDW);  ddw = fmaf(a1, xdd, ddw);
            WDD = __ffma2_rn(bc(c1), XW, WDD);   wdd = fmaf(c1, xw, wdd);
            DDp = __ffma2_rn(bc(b1), XD, DDp);   ddp = fmaf(b1, xd, ddp);
            if (WITH_G) {
                gWW = fmaf(a1, gW, gWW);
                gDW = fmaf(a1, gD, gDW);
                gWD = fmaf(b1, gW, gWD);
            }
        }
        const float a2 = w[2][k2], b2 = dw[2][k2], j2 = float(k2) * a2, jd2 = float(k2) * b2, c2 = dd[k2];
        V = __ffma2_rn(bc(a2), WW, V);                 v_ = fmaf(a2, ww, v_);
        M[0] = __ffma2_rn(bc(a2), JW, M[0]);           M_[0] = fmaf(a2, jw, M_[0]);
        M[1] = __ffma2_rn(bc(a2), WJ, M[1]);           M_[1] = fmaf(a2, wj, M_[1]);
        M[2] = __ffma2_rn(bc(j2), WW, M[2]);           M_[2] = fmaf(j2, ww, M_[2]);
        L[0] = __ffma2_rn(bc(a2), DW, L[0]);           L_[0] = fmaf(a2, dw_, L_[0]);
        L[1] = __ffma2_rn(bc(a2), WD, L[1]);           L_[1] = fmaf(a2, wd, L_[1]);
        L[2] = __ffma2_rn(bc(b2), WW, L[2]);           L_[2] = fmaf(b2, ww, L_[2]);
        Q[0][0] = __ffma2_rn(bc(a2), JDW, Q[0][0]);    Q_[0][0] = fmaf(a2, jdw, Q_[0][0]);
        Q[1][1] = __ffma2_rn(bc(a2), WJD, Q[1][1]);    Q_[1][1] = fmaf(a2, wjd, Q_[1][1]);
        Q[2][2] = __ffma2_rn(bc(jd2), WW, Q[2][2]);    Q_[2][2] = fmaf(jd2, ww, Q_[2][2]);
        Q[0][1] = __ffma2_rn(bc(a2), JD, Q[0][1]);     Q_[0][1] = fmaf(a2, jd, Q_[0][1]);
        Q[0][2] = __ffma2_rn(bc(b2), JW, Q[0][2]);     Q_[0][2] = fmaf(b2, jw, Q_[0][2]);
        Q[1][0] = __ffma2_rn(bc(a2), DJ, Q[1][0]);     Q_[1][0] = fmaf(a2, dj, Q_[1][0]);
        Q[1][2] = __ffma2_rn(bc(b2), WJ, Q[1][2]);     Q_[1][2] = fmaf(b2, wj, Q_[1][2]);
        Q[2][0] = __ffma2_rn(bc(j2), DW, Q[2][0]);     Q_[2][0] = fmaf(j2, dw_, Q_[2][0]);
        Q[2][1] = __ffma2_rn(bc(j2), WD, Q[2][1]);     Q_[2][1] = fmaf(j2, wd, Q_[2][1]);
        H[0] = __ffma2_rn(bc(a2), DDW, H[0]);          H_[0] = fmaf(a2, ddw, H_[0]);
        H[1] = __ffma2_rn(bc(a2), WDD, H[1]);          H_[1] = fmaf(a2, wdd, H_[1]);
        H[2] = __ffma2_rn(bc(c2), WW, H[2]);           H_[2] = fmaf(c2, ww, H_[2]);
        H[3] = __ffma2_rn(bc(a2), DDp, H[3]);          H_[3] = fmaf(a2, ddp, H_[3]);
        H[4] = __ffma2_rn(bc(b2), DW, H[4]);           H_[4] = fmaf(b2, dw_, H_[4]);
        H[5] = __ffma2_rn(bc(b2), WD, H[5]);           H_[5] = fmaf(b2, wd, H_[5]);
        if (WITH_G) {
            Lg[0] = fmaf(a2, gDW, Lg[0]);
            Lg[1] = fmaf(a2, gWD, Lg[1]);
            Lg[2] = fmaf(b2, gWW, Lg[2]);
        }
    }
    auto put = [](float *dst, float2 pr, float sc) {    // dst[c] for c = 0, 1, 2
        dst[PC] = pr.x;
        dst[PC + 1] = pr.y;
        dst[SC] = sc;
    };
    put(m.V, V, v_);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        put(m.M[b], M[b], M_[b]);
        put(m.L[b], L[b], L_[b]);
#pragma unroll
        for (int e = 0; e < 3; ++e) put(m.Q[e][b], Q[e][b], Q_[e][b]);
        m.Lg[b] = Lg[b];
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) put(m.H[q], H[q], H_[q]);
}

#ifndef MPM_ADJ_X2
#define MPM_ADJ_X2 1
#endif

__device__ __forceinline__ int hidx3(int b, int a)
{
    return b == a ? b : (b + a == 1 ? 3 : (b + a == 2 ? 4 : 5));
}

// 3D adjoint of G2P (same outputs as k_adj_g2p_bwd): the forward velocity
// moments and the x-derivatives of the weights enter through stencil moments of
// the node velocities; only the scatter of v_bar runs node by node.
template <class R, bool SPLIT>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? MPM_ADJ3_MINB : 1)
    k_adj_g2p_bwd3(const Params<R> P, const R *__restrict__ st, const R4<R> *__restrict__ GV,
                   const R *__restrict__ lam_in, R *__restrict__ lam_out, R4<R> *__restrict__ GVB,
                   R *__restrict__ coef)
{
    constexpr int D = 3, JC = 2 * D, JR = 2 * D + D * D;
    const int64_t n = P.n;
    const R cscale = R(4) * P.inv_dx;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        R x[D];
#pragma unroll
        for (int a = 0; a < D; ++a) x[a] = st[a * n + p];
        AdjStencil<R, D> s;
        adj_stencil<R, D>(P, x, s);
        Mom3<R> m;
        auto loadv = [&](int k0, int k1, int k2, R f[3], R &g) {
            const int a3[3] = {s.b[0] + 2 + k0, s.b[1] + 2 + k1, s.b[2] + 2 + k2};
            const R4<R> v4 = GV[lin3<D>(a3, P.G_nodes)];
            f[0] = v4.x;
            f[1] = v4.y;
            f[2] = v4.z;
            g = R(0);
        };
        if constexpr (sizeof(R) == 4 && MPM_ADJ_X2) stencil_moments3_x2<0, false>(s.w, s.dw, P.inv_dx, loadv, m);
        else stencil_moments3<R, false>(s.w, s.dw, P.inv_dx, loadv, m);
        R vp[D], Lf[D * D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            vp[a] = m.V[a];
#pragma unroll
            for (int b = 0; b < D; ++b) Lf[a * D + b] = m.L[b][a];
        }
        const R trL = Lf[0] + Lf[4] + Lf[8];
        R xb[D], vbt[D], Cb[D * D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const R xo = lam_in[a * n + p];
            const R xn = x[a] + P.dt * vp[a];
            const bool clamped = xn < R(0) || xn > P.L[a];
            xb[a] = clamped ? R(0) : xo;
            vbt[a] = lam_in[(D + a) * n + p] + (clamped ? R(0) : P.dt * xo);
        }
#pragma unroll
        for (int q = 0; q < D * D; ++q) Cb[q] = lam_in[(JC + q) * n + p];
        const R rho = st[JR * n + p];
        const R den = R(1) + P.dt * trL;
        const R rb1 = lam_in[JR * n + p];
        const R trLb = -rb1 * rho * P.dt / (den * den);
        R Lb[D * D];
#pragma unroll
        for (int q = 0; q < D * D; ++q) Lb[q] = (q % 4 == 0) ? trLb : R(0);
        if (P.material == 1) {
            R s6[6], sb6[6], s0b[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                s6[k] = st[(JR + 1 + k) * n + p];
                sb6[k] = lam_in[(JR + 1 + k) * n + p];
                s0b[k] = R(0);
            }
            dp_update_vjp<R>(P, Lf, s6, sb6, s0b, Lb);
#pragma unroll
            for (int k = 0; k < 6; ++k) lam_out[(JR + 1 + k) * n + p] = s0b[k];
        }
        // x through C's explicit fx: C = (4 / dx) sum w v (k - fx), dfx/dx = 1 / dx
#pragma unroll
        for (int b = 0; b < D; ++b) {
            R sacc = R(0);
#pragma unroll
            for (int a = 0; a < D; ++a) sacc += Cb[a * D + b] * vp[a];
            xb[b] -= cscale * P.inv_dx * sacc;
        }
        // x through the weights: sum_k wbar_k d_b w_k + sum_k d_b d_a w_k gbar_ka with
        // wbar_k = sum_a v_ka (vbt_a + cscale sum_c Cb_ac (k_c - fx_c)), gbar_ka = sum_d Lb_da v_kd
#pragma unroll
        for (int b = 0; b < D; ++b) {
            R acc = R(0);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                acc += vbt[a] * m.L[b][a];
#pragma unroll
                for (int c = 0; c < D; ++c)
                    acc += cscale * Cb[a * D + c] * (m.Q[c][b][a] - s.fx[c] * m.L[b][a]);
#pragma unroll
                for (int d = 0; d < D; ++d) acc += Lb[d * D + a] * m.H[hidx3(b, a)][d];
            }
            xb[b] += acc;
        }
        // v_bar scatter: v_bar_k = w_k (vbt + cscale Cb (k - fx)) + Lb grad w_k; with SPLIT
        // the coefficients (vbt, Cb, Lb) go to coef for the cell-ordered scatter pass
        if constexpr (SPLIT) {
#pragma unroll
            for (int a = 0; a < D; ++a) coef[a * n + p] = vbt[a];
#pragma unroll
            for (int q = 0; q < D * D; ++q) {
                coef[(3 + q) * n + p] = Cb[q];
                coef[(12 + q) * n + p] = Lb[q];
            }
        } else {
#pragma unroll
        for (int k = 0; k < 27; ++k) {
            const int kk[3] = {k % 3, (k / 3) % 3, k / 9};
            const R wy = s.w[1][kk[1]], wz = s.w[2][kk[2]], wx = s.w[0][kk[0]];
            const R w = wx * wy * wz;
            const R g[3] = {s.dw[0][kk[0]] * wy * wz, wx * s.dw[1][kk[1]] * wz, wx * wy * s.dw[2][kk[2]]};
            R vb[3];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                R cr = R(0), Lg = R(0);
#pragma unroll
                for (int b = 0; b < D; ++b) {
                    cr += Cb[a * D + b] * (R(kk[b]) - s.fx[b]);
                    Lg += Lb[a * D + b] * g[b];
                }
                vb[a] = w * (vbt[a] + cscale * cr) + Lg;
            }
            const int a3[3] = {s.b[0] + 2 + kk[0], s.b[1] + 2 + kk[1], s.b[2] + 2 + kk[2]};
            red_add4(&GVB[lin3<D>(a3, P.G_nodes)], vb[0], vb[1], vb[2], R(0));
        }
        }
#pragma unroll
        for (int a = 0; a < D; ++a) lam_out[a * n + p] = xb[a];
        lam_out[JR * n + p] = rb1 / den;
    }
}

// 3D adjoint of P2G (same outputs as k_adj_p2g_bwd) from stencil moments of the
// grid adjoint (P_bar as the three-component field, m_bar as the scalar one).
template <class R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? MPM_ADJ3P_MINB : 1)
    k_adj_p2g_bwd3(const Params<R> P, const R *__restrict__ st, const R4<R> *__restrict__ GAB,
                   R *__restrict__ lam_out)
{
    constexpr int D = 3, JV = D, JC = 2 * D, JR = 2 * D + D * D;
    const int64_t n = P.n;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        R x[D], v[D], C[D * D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            x[a] = st[a * n + p];
            v[a] = st[(JV + a) * n + p];
        }
#pragma unroll
        for (int q = 0; q < D * D; ++q) C[q] = st[(JC + q) * n + p];
        const R rho = st[JR * n + p];
        const R mp = P.mass;
        AdjStencil<R, D> s;
        adj_stencil<R, D>(P, x, s);
        Mom3<R> m;
        auto loadab = [&](int k0, int k1, int k2, R f[3], R &g) {
            const int a3[3] = {s.b[0] + 2 + k0, s.b[1] + 2 + k1, s.b[2] + 2 + k2};
            const R4<R> ab = GAB[lin3<D>(a3, P.G_nodes)];
            g = ab.x;
            f[0] = ab.y;
            f[1] = ab.z;
            f[2] = ab.w;
        };
        if constexpr (sizeof(R) == 4 && MPM_ADJ_X2) stencil_moments3_x2<1, true>(s.w, s.dw, P.inv_dx, loadab, m);
        else stencil_moments3<R, true>(s.w, s.dw, P.inv_dx, loadab, m);
        // stress-force coefficient Fm (P_a += Fm_ab d_b w)
        const bool sand = P.material == 1;
        R Fm[D * D];
        R pr = R(0);
        if (sand) {
            const R c = -P.dt * mp / rho;
            const int ix[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = 0; b < D; ++b) Fm[a * D + b] = c * st[(JR + 1 + ix[a][b]) * n + p];
        } else {
            pr = tait(P, rho);
            const R sforce = P.dt * mp / rho * pr;
#pragma unroll
            for (int q = 0; q < D * D; ++q) Fm[q] = (q % 4 == 0) ? sforce : R(0);
        }
        R xb[D];
#pragma unroll
        for (int b = 0; b < D; ++b) {
            R acc = mp * m.Lg[b];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                acc += mp * v[a] * m.L[b][a] - mp * C[a * D + b] * m.V[a];
#pragma unroll
                for (int c = 0; c < D; ++c)
                    acc += mp * C[a * D + c] * P.dx * (m.Q[c][b][a] - s.fx[c] * m.L[b][a]);
#pragma unroll
                for (int d = 0; d < D; ++d) acc += Fm[d * D + a] * m.H[hidx3(b, a)][d];
            }
            xb[b] = acc;
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            lam_out[a * n + p] += xb[a];
            lam_out[(JV + a) * n + p] = mp * m.V[a];
#pragma unroll
            for (int b = 0; b < D; ++b) lam_out[(JC + a * D + b) * n + p] = mp * P.dx * (m.M[b][a] - s.fx[b] * m.V[a]);
        }
        // adjoints of the stress and density through Fm (Fm_bar_ab = sum d_b w P_bar_a)
        if (sand) {
            const R c = -P.dt * mp / rho;
            R s6b[6] = {R(0), R(0), R(0), R(0), R(0), R(0)}, rhob = R(0);
            const int ix[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = 0; b < D; ++b) {
                    const R Fmb = m.L[b][a];
                    s6b[ix[a][b]] += c * Fmb;
                    rhob -= Fmb * Fm[a * D + b] / rho;
                }
            lam_out[JR * n + p] += rhob;
#pragma unroll
            for (int k = 0; k < 6; ++k) lam_out[(JR + 1 + k) * n + p] += s6b[k];
        } else {
            const R sb = m.L[0][0] + m.L[1][1] + m.L[2][2];
            const R r1 = rho * P.inv_rho0;
            R dp = P.bulk_K * P.inv_rho0;
            if (P.gamma_int > 0) {
                for (int k = 1; k < P.gamma_int; ++k) dp *= r1;
            } else {
                dp *= pow(r1, P.gamma - R(1));
            }
            const R dsdrho = P.dt * mp * (dp * rho - pr) / (rho * rho);
            lam_out[JR * n + p] += sb * dsdrho;
        }
    }
}

// ------------------------------------------------------------------ launchers

struct AdjDev {
    void *GVB, *GAB;                    // adjoint grid buffers (R4 per node)
    // 3D single precision: the v_bar scatter runs as a cell-ordered pass (k_p2g_direct,
    // MAT 2) when the sort tables of the state's generation are given
    void *coef = nullptr;               // 21 x n scatter coefficients
    int32_t *cursor = nullptr;          // its work-item cursor (zero between steps)
    const int4 *tiles = nullptr;        // sort tables of the state's generation
    const int32_t *n_tiles = nullptr, *posmap = nullptr, *cell_off = nullptr;
};

template <class R, int D> struct AdjLaunch {
    static int pblocks(const HostParams &h, const DevState &ds) { return grid_blocks(h.n, 256, ds.num_sms, 8); }
    static void save(const HostParams &h, DevState &ds, void *dst)
    {
        auto P = make_params<R>(h, ds);
        k_adj_save<R, D><<<pblocks(h, ds), 256, 0, ds.stream>>>(P, (const R *)ds.S, ds.id, (R *)dst);
    }
    static void restore(const HostParams &h, DevState &ds, const void *src)
    {
        auto P = make_params<R>(h, ds);
        k_adj_restore<R, D><<<pblocks(h, ds), 256, 0, ds.stream>>>(P, (R *)ds.S, ds.id, (const R *)src);
    }
    static void track(const HostParams &h, DevState &ds, const int32_t *track_of_id, double *out)
    {
        auto P = make_params<R>(h, ds);
        k_adj_track<R, D><<<pblocks(h, ds), 256, 0, ds.stream>>>(P, (const R *)ds.S, ds.id, track_of_id, out);
    }
    static void seed(const HostParams &h, DevState &ds, int n_track, const int64_t *ids, const double *x_obs,
                     const double *z_obs, void *lam)
    {
        k_adj_seed<R, D><<<(n_track + 255) / 256, 256, 0, ds.stream>>>(h.n, n_track, ids, x_obs, z_obs, (R *)lam);
    }
    static void reorder(const HostParams &h, DevState &ds, int nc, const int32_t *id_old, int32_t *pos_scratch,
                        const int32_t *id_new, const void *in, void *out)
    {
        k_adj_inverse<R><<<pblocks(h, ds), 256, 0, ds.stream>>>(h.n, id_old, pos_scratch);
        k_adj_reorder<R><<<pblocks(h, ds), 256, 0, ds.stream>>>(h.n, nc, pos_scratch, id_new, (const R *)in,
                                                                   (R *)out);
    }
    static void seed_slots(const HostParams &h, DevState &ds, const int32_t *id, const int32_t *track_of_id,
                           const double *x_obs, const double *z_obs, void *lam)
    {
        k_adj_seed_slots<R, D><<<pblocks(h, ds), 256, 0, ds.stream>>>(h.n, id, track_of_id, x_obs, z_obs, (R *)lam);
    }
    static void monitor_sum(const HostParams &h, DevState &ds, const void *x, const void *v, int64_t ld, int n_mon,
                            const double *boxes, double *sums)
    {
        k_monitor_sum<R, D><<<pblocks(h, ds), 256, 0, ds.stream>>>(h.n, ld, (const R *)x, (const R *)v, n_mon,
                                                                    boxes, sums);
    }
    static void monitor_seed(const HostParams &h, DevState &ds, const void *x, int64_t ld, int n_mon,
                             const double *boxes, const double *g, void *lam)
    {
        k_monitor_seed<R, D><<<pblocks(h, ds), 256, 0, ds.stream>>>(h.n, ld, (const R *)x, n_mon, boxes, g,
                                                                     (R *)lam);
    }
    static void gather(const HostParams &h, DevState &ds, int w, int off, const int32_t *id, const void *lam,
                       double *out)
    {
        k_adj_gather<R><<<pblocks(h, ds), 256, 0, ds.stream>>>(h.n, w, off, id, (const R *)lam, out);
    }
    static void scatter_in(const HostParams &h, DevState &ds, int w, int off, const int32_t *id, const double *in,
                           void *lam)
    {
        k_adj_scatter_in<R><<<pblocks(h, ds), 256, 0, ds.stream>>>(h.n, w, off, id, in, (R *)lam);
    }
    static void zero(DevState &ds, void *p, int64_t count)
    {
        k_adj_zero<R><<<grid_blocks(count, 256, ds.num_sms, 8), 256, 0, ds.stream>>>((R *)p, count);
    }
    // One reverse step: lam_in (adjoint of S^{t+1}) -> lam_out (adjoint of S^t) for the state st,
    // whose grid (m, q + dt f) and post-wall velocity the forward recompute saved in GA, GV.
    static void step(const HostParams &h, DevState &ds, const AdjDev &a, const void *st, const void *GA,
                     const void *GV, const int32_t *GL, const void *lam_in, void *lam_out, MuBar mub)
    {
        auto P = make_params<R>(h, ds);
        bool split = false;
        if constexpr (D == 3 && MPM_ADJ_SEPARABLE) {
            if constexpr (sizeof(R) == 4 && MPM_P2G_DIRECT) split = a.coef != nullptr && a.tiles != nullptr;
            if (split) {
                if constexpr (sizeof(R) == 4 && MPM_P2G_DIRECT) {
                    k_adj_g2p_bwd3<R, true><<<pblocks(h, ds), 256, 0, ds.stream>>>(
                        P, (const R *)st, (const R4<R> *)GV, (const R *)lam_in, (R *)lam_out, (R4<R> *)a.GVB,
                        (R *)a.coef);
                    constexpr int NT = 128;
                    constexpr size_t smem = p2g_direct_smem<R, 3, NT, 2>();
                    static_assert(smem <= 48 * 1024, "k_p2g_direct shared memory above the default limit");
                    P2GIO<R> io{(const R *)st, (const R *)a.coef, h.n, a.tiles, a.n_tiles, a.cursor, a.posmap,
                                a.cell_off, (R4<R> *)a.GVB, nullptr};
                    k_p2g_direct<R, 3, NT, 2><<<ds.num_sms * MPM_P2G_MINB, NT, smem, ds.stream>>>(P, io, nullptr,
                                                                                               nullptr);
                }
            } else {
                k_adj_g2p_bwd3<R, false><<<pblocks(h, ds), 256, 0, ds.stream>>>(
                    P, (const R *)st, (const R4<R> *)GV, (const R *)lam_in, (R *)lam_out, (R4<R> *)a.GVB, nullptr);
            }
        } else {
            k_adj_g2p_bwd<R, D><<<pblocks(h, ds), 256, 0, ds.stream>>>(P, (const R *)st, (const R4<R> *)GV,
                                                                         (const R *)lam_in, (R *)lam_out,
                                                                         (R4<R> *)a.GVB);
        }
        int64_t nbg = h.node_tiles_per_sim;             // blocks stride the saved tile list
        if (nbg > (int64_t)ds.num_sms * 8) nbg = (int64_t)ds.num_sms * 8;
        k_adj_grid_bwd<R, D><<<(unsigned)nbg, 256, 0, ds.stream>>>(P, (const R4<R> *)GA, (R4<R> *)a.GVB,
                                                                   (R4<R> *)a.GAB, GL, mub,
                                                                   split ? a.cursor : nullptr);
        if constexpr (D == 3 && MPM_ADJ_SEPARABLE)
            k_adj_p2g_bwd3<R><<<pblocks(h, ds), 256, 0, ds.stream>>>(P, (const R *)st, (const R4<R> *)a.GAB,
                                                                   (R *)lam_out);
        else
            k_adj_p2g_bwd<R, D><<<pblocks(h, ds), 256, 0, ds.stream>>>(P, (const R *)st, (const R4<R> *)a.GAB,
                                                                         (R *)lam_out);
    }
};

template <class R> struct AdjDispatch {
#define MPM_ADJ_DISPATCH(name, args, call)                   \
    static void name args                                    \
    {                                                        \
        if (h.dim == 2) AdjLaunch<R, 2>::call;               \
        else AdjLaunch<R, 3>::call;                          \
    }
    MPM_ADJ_DISPATCH(save, (const HostParams &h, DevState &ds, void *dst), save(h, ds, dst))
    MPM_ADJ_DISPATCH(restore, (const HostParams &h, DevState &ds, const void *src), restore(h, ds, src))
    MPM_ADJ_DISPATCH(track, (const HostParams &h, DevState &ds, const int32_t *t, double *o), track(h, ds, t, o))
    MPM_ADJ_DISPATCH(seed, (const HostParams &h, DevState &ds, int nt, const int64_t *ids, const double *xo,
                            const double *zo, void *lam), seed(h, ds, nt, ids, xo, zo, lam))
    MPM_ADJ_DISPATCH(step, (const HostParams &h, DevState &ds, const AdjDev &a, const void *st, const void *ga,
                            const void *gv, const int32_t *gl, const void *li, void *lo, MuBar mub),
                     step(h, ds, a, st, ga, gv, gl, li, lo, mub))
    MPM_ADJ_DISPATCH(reorder, (const HostParams &h, DevState &ds, int nc, const int32_t *id_old, int32_t *pos,
                               const int32_t *id_new, const void *in, void *out),
                     reorder(h, ds, nc, id_old, pos, id_new, in, out))
    MPM_ADJ_DISPATCH(seed_slots, (const HostParams &h, DevState &ds, const int32_t *id, const int32_t *tid,
                                  const double *xo, const double *zo, void *lam), seed_slots(h, ds, id, tid, xo, zo, lam))
    MPM_ADJ_DISPATCH(monitor_sum, (const HostParams &h, DevState &ds, const void *x, const void *v, int64_t ld,
                                   int nm, const double *b, double *s), monitor_sum(h, ds, x, v, ld, nm, b, s))
    MPM_ADJ_DISPATCH(monitor_seed, (const HostParams &h, DevState &ds, const void *x, int64_t ld, int nm,
                                    const double *b, const double *g, void *lam),
                     monitor_seed(h, ds, x, ld, nm, b, g, lam))
    MPM_ADJ_DISPATCH(gather, (const HostParams &h, DevState &ds, int w, int off, const int32_t *id, const void *lam,
                              double *out), gather(h, ds, w, off, id, lam, out))
    MPM_ADJ_DISPATCH(scatter_in, (const HostParams &h, DevState &ds, int w, int off, const int32_t *id,
                                  const double *in, void *lam), scatter_in(h, ds, w, off, id, in, lam))
#undef MPM_ADJ_DISPATCH
    static void zero(const HostParams &, DevState &ds, void *p, int64_t count) { AdjLaunch<R, 2>::zero(ds, p, count); }
};

}  // namespace mpm
