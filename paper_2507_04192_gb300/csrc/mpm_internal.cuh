// Internal definitions of libmpm shared by its translation units.
//
// Grid geometry.  A physical node j (0 <= j <= N + 2 per axis) sits at
// (j - 1) dx: one ghost node below the wall at 0 and one beyond the wall at
// L = N dx (Sec. 2.2, ghost cells).  The device arrays use the shifted index
// a = j + 1, with one extra pad node below so that the shared-memory window
// of every tile starts at a non-negative index.  A particle's first stencil
// node ("base") is s = floor(x / dx - 0.5) + 2 in a-space, s in [1, N + 1].
// Particles are grouped by the tile of their base node: tile t covers
// s in [t T + 1, t T + T] (a-space) at sort time, and its window covers the
// nodes [t T, t T + T + 4), which holds the 3^d stencil of any particle whose
// base has moved at most one node since the sort.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace mpm {

constexpr int kMaxWalls = 6;
constexpr int kMaxObstacles = 8;

// Stationary box obstacles in node units: a node with integer coordinate c
// (position c dx) is inside when lo[a] <= c[a] <= hi[a] on every axis; bit 2a
// (2a + 1) of faces is set when the low (high) face of axis a is a contact face.
struct Obstacles {
    int n;
    int lo[kMaxObstacles][3], hi[kMaxObstacles][3];
    int faces[kMaxObstacles];
};
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortChunk = kSortThreads * kSortItems;
constexpr int kScanSegments = 1024;              // scratch words after the digit histogram

// Particle state layout: blocks of kPB particles (the slots 32 b .. 32 b + 31);
// inside a block the components follow each other, component c of the block's
// particle r at element c kPB + r.  All components of one particle therefore sit
// at fixed offsets (multiples of kPB elements) from one address, and a warp that
// reads one component of kPB consecutive particles reads one contiguous line.
constexpr int kPB = 32;
// First element of particle p's components (component c at + c kPB).
__host__ __device__ __forceinline__ int64_t sblock(int64_t p, int ncomp)
{
    return (p >> 5) * (int64_t)ncomp * kPB + (p & (kPB - 1));
}
// Element of component c of particle i in a state view: component-major with
// stride ld (ld > 0) or blocked as above with -ld components (ld < 0).
template <class R> __host__ __device__ __forceinline__ R sview(const R *base, int64_t ld, int c, int64_t i)
{
    return ld > 0 ? base[c * ld + i] : base[sblock(i, (int)(-ld)) + (int64_t)c * kPB];
}

template <int D> struct Geo;
template <> struct Geo<2> {
    static constexpr int T = 16;                 // cells per tile edge
    static constexpr int W = T + 4;              // window edge (nodes)
    static constexpr int WN = W * W;             // window nodes
    static constexpr int TN = T * T;             // cells per tile
    static constexpr int CELL_BITS = 8;          // log2(TN)
    static constexpr int STENCIL = 9;
    static constexpr int NG = 256;               // cells per group (= threads of a P2G block)
};
template <> struct Geo<3> {
    static constexpr int T = 8;
    static constexpr int W = T + 4;
    static constexpr int WN = W * W * W;
    static constexpr int TN = T * T * T;
    static constexpr int CELL_BITS = 9;
    static constexpr int STENCIL = 27;
    static constexpr int NG = 64;                // cells per group: one 8 x 8 layer of the tile
};

// Friction field of one wall on the device.
struct WallDev {
    int n_seg[2];
    int seg_axis[2];       // tangential axes
    const void *mu;        // batch x n_seg1 x n_seg0 reals (R), nullptr = slip
};

// Host-side parameters (double), converted to Params<R> at launch.
struct HostParams {
    int dim, batch, precision, material, dp_literal, transfer;
    double flip_alpha;
    int n_cells[3];
    double dx, dt, gravity[3];
    double rho0, bulk_K, gamma, mass, vol0, m_eps;
    double K, G, q_phi, k_phi, q_psi, sig_t, tau_P, alpha_P;
    int T, W, n_tiles[3], G_nodes[3], node_tiles[3];
    int64_t nodes_per_sim, tiles_per_sim, node_tiles_per_sim;
    int64_t n, npad;
    int ncomp, off_x, off_v, off_C, off_F, off_rho, off_sig, off_eps;
    Obstacles obs;
    int debug;                    // kDebug* bits (test hooks of the error paths)
};

template <class R>
struct Params {
    int n_cells[3];
    R dx, inv_dx, dt, gravity[3], L[3];
    R rho0, bulk_K, gamma, inv_rho0, mass, m_eps, K_over_gamma;
    R K, G, q_phi, k_phi, q_psi, sig_t, tau_P, alpha_P, eps2_coef, inv_G_Kqq, inv_K;
    int material, dp_literal, gamma_int, transfer, no_force;
    R flip_alpha;
    R *save_S;                    // P2G: copy of its inputs in slot order (nullptr = none)
    uint32_t *flags;              // node tile flags, the touched-tile list and its length
    int32_t *node_list, *list_count;
    int n_tiles[3], G_nodes[3], node_tiles[3];
    int64_t nodes_per_sim, tiles_per_sim, node_tiles_per_sim;
    int64_t n, npad;
    int ncomp, off_x, off_v, off_C, off_F, off_rho, off_sig, off_eps;
    WallDev wall[kMaxWalls];
    Obstacles obs;
    double *diag;                 // conservation sums of the step (nullptr = off), see kDiag*
    int debug;
};

template <class R> struct R4 { R x, y, z, w; };
template <> struct alignas(16) R4<float> { float x, y, z, w; };
template <> struct alignas(32) R4<double> { double x, y, z, w; };

// Device pointers and launch state of one context.
struct DevState {
    cudaStream_t stream;
    int num_sms;
    void *S, *S2;                 // particle state, ncomp x npad reals in blocks of kPB particles (sblock)
    int32_t *id, *id2;            // load-order id of each sorted slot
    int32_t *sim, *sim2;          // simulation id of each slot
    uint32_t *keys[2];
    int32_t *vals[2];
    uint32_t *hist;               // kRadixBins x n_sort_blocks
    int32_t *tile_start, *tile_end;   // per tile (batch x tiles_per_sim)
    int4 *tiles;                  // compact non-empty tiles: (tile key, start, count, 0) in key order,
                                  // then (at + max_tiles) the same tiles largest first (G2P order)
    int64_t max_tiles;
    int32_t *perm;                // gather permutation of the last sort
    int32_t *posmap;              // per particle in (cell, rank) order: its slot relative to the tile start
    int32_t *cell_off;            // per compact tile: TN + 1 exclusive prefix sums of the cell counts
    int32_t *counters;            // [1] n_active_tiles, [2] P2G tile cursor, [3] G2P tile cursor,
                                  // [4] length of the touched node-tile list
    void *A, *V;                  // grid accumulators and velocities, R4 per node
    uint32_t *flags;              // per node tile: touched since the last grid update
    int32_t *node_list;           // the touched node tiles, in the order P2G touched them
    int32_t *status;              // device status word (bit 0: non-finite state)
    unsigned long long *escaped;  // particles that took the out-of-window path
    double *staging;              // n x 9 doubles for host transfers
    void *A2 = nullptr, *V2 = nullptr;   // FLIP: (m, q) without forces and the pre-update grid velocity
    void *save_A = nullptr;       // when set, the grid update also copies (m, q + dt f) ...
    void *save_V = nullptr;       // ... and the post-wall velocity of every node it updates here,
    int32_t *save_L = nullptr;    // ... and the list of node tiles it updated ([0] count, then the tiles)
    void *save_S = nullptr;       // when set, P2G copies the components it reads (x, v, C, rho [, sigma])
                                  // of every particle here, in slot order (save_S[c n + slot])
    double *diag = nullptr;       // kDiagCount doubles: conservation sums of the last step (when enabled)
    CUtensorMap tmap_V;           // TMA descriptor of V: (4, G_x, G_y, [G_z], batch)
    void *mu_dev[kMaxWalls];
    int n_seg[kMaxWalls][2];
    int key_bits;
};

enum StatusBits { kStatusNaN = 1, kStatusChunkOverflow = 2, kStatusTimeout = 4 };

// Test hooks (HostParams::debug): kDebugWithholdWindowCopy makes G2P arm no copy
// for its grid window, so that its bounded wait runs out with nothing in flight.
enum DebugBits { kDebugWithholdWindowCopy = 1 };

// Slots of the conservation sums (DevState::diag), all in double precision:
// grid mass, grid momentum (3), particle mass, particle momentum (3), non-finite
// grid values, non-finite particle values, sum of |momentum components| on the grid.
enum DiagSlots {
    kDiagGridMass = 0, kDiagGridMom = 1, kDiagPartMass = 4, kDiagPartMom = 5, kDiagGridNonFinite = 8,
    kDiagPartNonFinite = 9, kDiagGridAbsMom = 10, kDiagCount = 11
};

// Launchers implemented per precision (mpm_kernels_f32.cu, mpm_kernels_f64.cu).
struct Ops {
    void (*init_state)(const HostParams &, DevState &, const double *x_dev, const double *v_dev);
    void (*keys)(const HostParams &, DevState &);
    void (*permute)(const HostParams &, DevState &);
    void (*p2g)(const HostParams &, DevState &);
    void (*grid)(const HostParams &, DevState &);
    void (*g2p)(const HostParams &, DevState &);
    void (*get_field)(const HostParams &, DevState &, int field, double *out_dev);
    void (*set_field)(const HostParams &, DevState &, int field, const double *in_dev);
    void (*diag_particles)(const HostParams &, DevState &);
};
extern const Ops ops_f32;
extern const Ops ops_f64;

struct AdjDev;
struct MuBar;
// Adjoint launchers per precision.
struct AdjOps {
    void (*save)(const HostParams &, DevState &, void *dst);
    void (*restore)(const HostParams &, DevState &, const void *src);
    void (*track)(const HostParams &, DevState &, const int32_t *track_of_id, double *out);
    void (*seed)(const HostParams &, DevState &, int n_track, const int64_t *ids, const double *x_obs,
                 const double *z_obs, void *lam);
    void (*step)(const HostParams &, DevState &, const AdjDev &, const void *st, const void *GA, const void *GV,
                 const int32_t *GL, const void *lam_in, void *lam_out, MuBar mub);
    void (*zero)(const HostParams &, DevState &, void *p, int64_t count);
    void (*reorder)(const HostParams &, DevState &, int nc, const int32_t *id_old, int32_t *pos_scratch,
                    const int32_t *id_new, const void *in, void *out);
    void (*seed_slots)(const HostParams &, DevState &, const int32_t *id, const int32_t *track_of_id,
                       const double *x_obs, const double *z_obs, void *lam);
    // velocity monitors: sums of v and counts per box; the adjoint seed of their loss
    void (*monitor_sum)(const HostParams &, DevState &, const void *x, const void *v, int64_t ld, int n_mon,
                        const double *boxes, double *sums);
    void (*monitor_seed)(const HostParams &, DevState &, const void *x, int64_t ld, int n_mon,
                         const double *boxes, const double *g, void *lam);
    // out[id[s] w + k] = lam[(off + k) n + s]
    void (*gather)(const HostParams &, DevState &, int w, int off, const int32_t *id, const void *lam, double *out);
    // lam[(off + k) n + s] = in[id[s] w + k]
    void (*scatter_in)(const HostParams &, DevState &, int w, int off, const int32_t *id, const double *in,
                       void *lam);
};
constexpr int kMaxMonitors = 64;
extern const AdjOps adj_ops_f32;
extern const AdjOps adj_ops_f64;

// Sort helpers (mpm_sort.cu), precision independent.
void radix_sort_pairs(const HostParams &hp, DevState &ds);
void build_tiles(const HostParams &hp, DevState &ds);

}  // namespace mpm
