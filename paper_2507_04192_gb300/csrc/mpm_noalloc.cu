// mpm_step_noalloc: one explicit MPM step that allocates no memory.
//
// Some callers cannot call cudaMalloc: plugins hosted by an application that
// owns all device memory and forbids others from allocating, and real-time
// loops that must not hit the allocator's latency (cudaMalloc may synchronise
// the device) or its failure modes.  For them this entry point takes the particle state in and
// out through caller-owned device buffers and keeps its only scratch -- the
// background grid -- in the file-scope device array below.  It performs no
// allocation of its own: no cudaMalloc, cudaFree, context, stream or library
// call that allocates.
//
// The grid scratch is shared by every call on a device and keeps the last
// call's contents; each call clears it before use.  Calls whose work overlaps
// on the GPU (two streams, or two host threads) race on it: serialise them.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/mpm.h"
#include "mpm_kernels.cuh"

namespace {

// Grid scratch: 4 doubles per node (mass, then momentum; velocity in place).
constexpr int64_t kNoallocMaxNodes = int64_t(1) << 17;            // 4 MiB
static __device__ __align__(256) double na_grid[kNoallocMaxNodes * 4];

std::mutex na_mutex;
constexpr int kMaxDevices = 64;
double *na_grid_addr[kMaxDevices] = {nullptr};

using mpm::Params;

struct NaDims {
    int d;
    int N[3];
    int G[3];            // nodes per axis (N + 3), node j at (j - 1) dx
    int64_t nodes;
};

__device__ __forceinline__ int64_t na_node(const NaDims &g, const int j[3])
{
    int64_t idx = 0;
    for (int a = g.d - 1; a >= 0; --a) idx = idx * g.G[a] + j[a];
    return idx;
}

__global__ void k_na_clear(double *grid, int64_t count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        grid[i] = 0.0;
}

// P2G with direct double atomics into the scratch grid (no sort).
__global__ void k_na_p2g(const Params<double> P, NaDims g, int64_t n, mpm_state_ptrs in, double *grid)
{
    const int d = g.d;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        double x[3] = {0, 0, 0}, v[3] = {0, 0, 0}, C[9] = {0}, S[9] = {0};
        for (int a = 0; a < d; ++a) {
            x[a] = in.x[p * d + a];
            v[a] = in.v[p * d + a];
        }
        for (int q = 0; q < d * d; ++q) C[q] = in.C[p * d * d + q];
        const double rho = in.rho[p];
        const double Vp = P.mass / rho;
        if (P.material == 0) {
            const double pr = mpm::tait(P, rho);
            for (int a = 0; a < 3; ++a) S[a * 3 + a] = -pr;
        } else {
            for (int q = 0; q < 9; ++q) S[q] = in.sigma[p * 9 + q];
        }
        int b[3] = {0, 0, 0};
        double fx[3] = {0, 0, 0}, w[3][3] = {{0}}, dw[3][3] = {{0}};
        for (int a = 0; a < d; ++a) {
            b[a] = mpm::base_cell(x[a], P.inv_dx, g.N[a]);
            fx[a] = x[a] * P.inv_dx - b[a];
            mpm::bspline(fx[a], P.inv_dx, w[a], dw[a]);
        }
        const int nk = d == 2 ? 9 : 27;
        for (int k = 0; k < nk; ++k) {
            const int kk[3] = {k % 3, (k / 3) % 3, k / 9};
            double wt = 1.0, gr[3] = {1.0, 1.0, 1.0};
            int j[3] = {0, 0, 0};
            for (int a = 0; a < d; ++a) {
                j[a] = b[a] + 1 + kk[a];
                wt *= w[a][kk[a]];
                for (int c = 0; c < d; ++c) gr[c] *= (c == a) ? dw[a][kk[a]] : w[a][kk[a]];
            }
            double *node = grid + na_node(g, j) * 4;
            atomicAdd(&node[0], P.mass * wt);
            for (int a = 0; a < d; ++a) {
                double aff = v[a];
                for (int c = 0; c < d; ++c) aff += C[a * d + c] * (kk[c] - fx[c]) * P.dx;
                double f = 0.0;
                for (int c = 0; c < d; ++c) f += S[a * 3 + c] * gr[c];
                atomicAdd(&node[1 + a], P.mass * wt * aff - P.dt * Vp * f);
            }
        }
    }
}

// Grid update in place: velocity from momentum, gravity, slip walls.
__global__ void k_na_grid(const Params<double> P, NaDims g, double *grid)
{
    const int d = g.d;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.nodes; i += (int64_t)gridDim.x * blockDim.x) {
        double *node = grid + i * 4;
        const double m = node[0];
        double vel[3] = {0, 0, 0};
        if (m > P.m_eps)
            for (int a = 0; a < d; ++a) vel[a] = node[1 + a] / m + P.dt * P.gravity[a];
        int64_t r = i;
        for (int a = 0; a < d; ++a) {
            const int j = (int)(r % g.G[a]);
            r /= g.G[a];
            const int c = j - 1;                          // node coordinate / dx
            if (c <= 0 && vel[a] < 0.0) vel[a] = 0.0;     // low wall, outward normal -e_a
            if (c >= g.N[a] && vel[a] > 0.0) vel[a] = 0.0;
        }
        for (int a = 0; a < d; ++a) node[1 + a] = vel[a];
    }
}

// G2P from the scratch grid into the caller's output state.
__global__ void k_na_g2p(const Params<double> P, NaDims g, int64_t n, mpm_state_ptrs in, mpm_state_ptrs out,
                         const double *grid)
{
    const int d = g.d;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        double x[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) x[a] = in.x[p * d + a];
        int b[3] = {0, 0, 0};
        double fx[3] = {0, 0, 0}, w[3][3] = {{0}}, dw[3][3] = {{0}};
        for (int a = 0; a < d; ++a) {
            b[a] = mpm::base_cell(x[a], P.inv_dx, g.N[a]);
            fx[a] = x[a] * P.inv_dx - b[a];
            mpm::bspline(fx[a], P.inv_dx, w[a], dw[a]);
        }
        double vp[3] = {0, 0, 0}, Bm[9] = {0}, L[9] = {0};
        const int nk = d == 2 ? 9 : 27;
        for (int k = 0; k < nk; ++k) {
            const int kk[3] = {k % 3, (k / 3) % 3, k / 9};
            double wt = 1.0, gr[3] = {1.0, 1.0, 1.0};
            int j[3] = {0, 0, 0};
            for (int a = 0; a < d; ++a) {
                j[a] = b[a] + 1 + kk[a];
                wt *= w[a][kk[a]];
                for (int c = 0; c < d; ++c) gr[c] *= (c == a) ? dw[a][kk[a]] : w[a][kk[a]];
            }
            const double *node = grid + na_node(g, j) * 4;
            for (int a = 0; a < d; ++a) {
                const double vi = node[1 + a];
                vp[a] += wt * vi;
                for (int c = 0; c < d; ++c) {
                    Bm[a * d + c] += wt * vi * (kk[c] - fx[c]);
                    L[a * d + c] += vi * gr[c];
                }
            }
        }
        double trL = 0.0;
        for (int a = 0; a < d; ++a) trL += L[a * d + a];
        for (int a = 0; a < d; ++a) {
            double xn = x[a] + P.dt * vp[a];
            xn = xn < 0.0 ? 0.0 : (xn > P.L[a] ? P.L[a] : xn);
            out.v[p * d + a] = vp[a];
            out.x[p * d + a] = xn;
        }
        for (int q = 0; q < d * d; ++q) out.C[p * d * d + q] = Bm[q] * 4.0 * P.inv_dx;
        double F[9], Fn[9];
        for (int q = 0; q < d * d; ++q) F[q] = in.F[p * d * d + q];
        for (int a = 0; a < d; ++a)
            for (int c = 0; c < d; ++c) {
                double s = 0.0;
                for (int k = 0; k < d; ++k) s += L[a * d + k] * F[k * d + c];
                Fn[a * d + c] = F[a * d + c] + P.dt * s;
            }
        for (int q = 0; q < d * d; ++q) out.F[p * d * d + q] = Fn[q];
        const double rho = in.rho[p] / (1.0 + P.dt * trL);
        out.rho[p] = rho;
        if (P.material == 1) {
            double L3[9] = {0};
            for (int a = 0; a < d; ++a)
                for (int c = 0; c < d; ++c) L3[a * 3 + c] = L[a * d + c];
            const double *s9 = in.sigma + p * 9;
            double s6[6] = {s9[0], s9[4], s9[8], 0.5 * (s9[1] + s9[3]), 0.5 * (s9[2] + s9[6]), 0.5 * (s9[5] + s9[7])};
            double e = in.eps[p];
            mpm::dp_update(P, L3, s6, e);
            double *o9 = out.sigma + p * 9;
            o9[0] = s6[0]; o9[4] = s6[1]; o9[8] = s6[2];
            o9[1] = o9[3] = s6[3];
            o9[2] = o9[6] = s6[4];
            o9[5] = o9[7] = s6[5];
            out.eps[p] = e;
        }
    }
}

int set_msg(char *err, int err_len, const char *msg)
{
    if (err && err_len > 0) std::snprintf(err, (size_t)err_len, "%s", msg);
    return 0;
}

}  // namespace

extern "C" int mpm_step_noalloc(const mpm_grid_desc *grid, const mpm_material *material, void *cuda_stream,
                                int64_t n, double particle_volume, mpm_state_ptrs in, mpm_state_ptrs out,
                                char *err, int err_len)
{
    if (!grid || !material || n <= 0 || !(particle_volume > 0)) {
        set_msg(err, err_len, "mpm_step_noalloc: bad argument");
        return MPM_EINVAL;
    }
    const mpm_grid_desc &gd = *grid;
    const mpm_material &m = *material;
    if ((gd.dim != 2 && gd.dim != 3) || gd.precision != MPM_FP64 || gd.batch != 1 ||
        gd.transfer != MPM_TRANSFER_APIC || !(gd.dx > 0) ||
        !(gd.dt > 0) || (m.kind != MPM_FLUID && m.kind != MPM_DRUCKER_PRAGER) || !(m.rho0 > 0) ||
        (m.kind == MPM_FLUID && (m.viscosity != 0.0 || !(m.bulk_K > 0) || !(m.gamma > 0)))) {
        set_msg(err, err_len, "mpm_step_noalloc: needs dim 2 or 3, MPM_FP64, batch 1, APIC and a valid material");
        return MPM_EINVAL;
    }
    bool finite = std::isfinite(gd.dx) && std::isfinite(gd.dt) && std::isfinite(m.rho0);
    for (int a = 0; a < gd.dim; ++a) finite = finite && std::isfinite(gd.gravity[a]);
    if (m.kind == MPM_FLUID) finite = finite && std::isfinite(m.bulk_K) && std::isfinite(m.gamma);
    else
        finite = finite && m.E > 0.0 && std::isfinite(m.E) && m.nu > -1.0 && m.nu < 0.5 && m.phi_deg >= 0.0 &&
                 m.phi_deg < 90.0 && m.psi_deg >= 0.0 && m.psi_deg < 90.0 && m.cohesion >= 0.0 &&
                 std::isfinite(m.cohesion) && m.sigma_t >= 0.0 && std::isfinite(m.sigma_t);
    if (!finite) {
        set_msg(err, err_len, "mpm_step_noalloc: non-finite or out-of-range grid or material parameter");
        return MPM_EINVAL;
    }
    if (!in.x || !in.v || !in.C || !in.F || !in.rho || !out.x || !out.v || !out.C || !out.F || !out.rho ||
        (m.kind == MPM_DRUCKER_PRAGER && (!in.sigma || !in.eps || !out.sigma || !out.eps))) {
        set_msg(err, err_len, "mpm_step_noalloc: missing state buffer");
        return MPM_EINVAL;
    }
    NaDims g{};
    g.d = gd.dim;
    g.nodes = 1;
    for (int a = 0; a < 3; ++a) {
        g.N[a] = a < gd.dim ? gd.n_cells[a] : 1;
        g.G[a] = a < gd.dim ? g.N[a] + 3 : 1;
        if (a < gd.dim && (g.N[a] < 1 || g.N[a] > 4096)) {
            set_msg(err, err_len, "mpm_step_noalloc: cell count out of range");
            return MPM_EINVAL;
        }
        g.nodes *= g.G[a];
    }
    if (g.nodes > kNoallocMaxNodes) {
        char msg[160];
        std::snprintf(msg, sizeof msg,
                      "mpm_step_noalloc: grid of %lld nodes exceeds the maximum of %lld nodes of the static scratch",
                      (long long)g.nodes, (long long)kNoallocMaxNodes);
        set_msg(err, err_len, msg);
        return MPM_EINVAL;
    }
    // resolve the scratch array's device address once per device (host code
    // cannot pass the symbol itself to a kernel)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_msg(err, err_len, "mpm_step_noalloc: no current CUDA device");
        return MPM_ECUDA;
    }
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(na_mutex);
        if (!na_grid_addr[dev]) {
            double *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress((void **)&ptr, na_grid);
            if (e != cudaSuccess || ptr == nullptr) {
                set_msg(err, err_len, "mpm_step_noalloc: cudaGetSymbolAddress of the scratch grid failed");
                return MPM_ECUDA;
            }
            // load the four kernels now: with lazy module loading a kernel's code is
            // otherwise loaded (and device memory taken for it) at its first launch
            cudaFuncAttributes fa;
            const void *kernels[4] = {(const void *)k_na_clear, (const void *)k_na_p2g, (const void *)k_na_grid,
                                      (const void *)k_na_g2p};
            for (const void *k : kernels)
                if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
            if (e != cudaSuccess) {
                set_msg(err, err_len, "mpm_step_noalloc: loading the kernels failed");
                return MPM_ECUDA;
            }
            na_grid_addr[dev] = ptr;
        }
        scratch = na_grid_addr[dev];
    }
    mpm::HostParams h{};
    h.dim = gd.dim;
    h.batch = 1;
    h.precision = MPM_FP64;
    h.material = m.kind;
    h.dp_literal = m.dp_literal ? 1 : 0;
    h.dx = gd.dx;
    h.dt = gd.dt;
    for (int a = 0; a < 3; ++a) {
        h.n_cells[a] = g.N[a];
        h.gravity[a] = a < gd.dim ? gd.gravity[a] : 0.0;
    }
    h.rho0 = m.rho0;
    h.bulk_K = m.bulk_K;
    h.gamma = m.gamma;
    h.mass = m.rho0 * particle_volume;
    h.m_eps = 1e-10 * m.rho0 * std::pow(gd.dx, gd.dim);
    if (m.kind == MPM_DRUCKER_PRAGER) {
        const double pi = 3.14159265358979323846;
        const double phi = m.phi_deg * pi / 180.0, psi = m.psi_deg * pi / 180.0;
        h.K = m.E / (3.0 * (1.0 - 2.0 * m.nu));
        h.G = m.E / (2.0 * (1.0 + m.nu));
        h.q_phi = 6.0 * std::sin(phi) / (std::sqrt(3.0) * (3.0 + std::sin(phi)));
        h.k_phi = 6.0 * m.cohesion * std::cos(phi) / (std::sqrt(3.0) * (3.0 + std::sin(phi)));
        h.q_psi = 6.0 * std::sin(psi) / (std::sqrt(3.0) * (3.0 + std::sin(psi)));
        h.sig_t = m.sigma_t;
        if (h.q_phi > 0.0 && h.k_phi / h.q_phi < h.sig_t) h.sig_t = h.k_phi / h.q_phi;
        h.tau_P = h.k_phi - h.q_phi * h.sig_t;
        h.alpha_P = std::sqrt(1.0 + h.q_phi * h.q_phi) - h.q_phi;
    }
    mpm::DevState ds{};
    const Params<double> P = mpm::make_params<double>(h, ds);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const int threads = 256;
    const int nb_p = (int)((n + threads - 1) / threads < 4096 ? (n + threads - 1) / threads : 4096);
    const int nb_g = (int)((g.nodes + threads - 1) / threads < 4096 ? (g.nodes + threads - 1) / threads : 4096);
    k_na_clear<<<nb_g, threads, 0, stream>>>(scratch, g.nodes * 4);
    k_na_p2g<<<nb_p, threads, 0, stream>>>(P, g, n, in, scratch);
    k_na_grid<<<nb_g, threads, 0, stream>>>(P, g, scratch);
    k_na_g2p<<<nb_p, threads, 0, stream>>>(P, g, n, in, out, scratch);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "mpm_step_noalloc: launch failed: %s", cudaGetErrorString(e));
        set_msg(err, err_len, msg);
        return MPM_ECUDA;
    }
    set_msg(err, err_len, "");
    return MPM_OK;
}
