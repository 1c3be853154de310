// Host side of libmpm: context lifetime, device memory, the step sequence
// and the C-ABI declared in include/mpm.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/mpm.h"
#include "mpm_adjoint.cuh"

// Reverse sweep of one segment overlapped with the recompute of the one before it.
#ifndef MPM_ADJ_OVERLAP
#define MPM_ADJ_OVERLAP 1
#endif

using namespace mpm;
static_assert(MPM_DIAG_COUNT == kDiagCount, "diagnostics slots");

struct PendingTiming {
    int kernel;
    cudaEvent_t start, stop;
};

// Adjoint (reverse sweep) buffers and observations, allocated on first use.
struct AdjHost {
    int n_track = 0, n_obs = 0;
    std::vector<int64_t> ids;
    std::vector<int> steps;
    std::vector<double> z;                     // n_obs x n_track x dim
    int64_t *d_ids = nullptr;
    int32_t *d_track_of_id = nullptr;
    double *d_z = nullptr, *d_xobs = nullptr;
    void *ckpt = nullptr;
    int64_t ckpt_cap = 0;
    void *seg = nullptr;
    int64_t seg_cap = 0;
    void *seg_grid = nullptr;                  // per segment state: (m, q + dt f) and v of its step
    int64_t seg_grid_cap = 0;
    int32_t *seg_id = nullptr;                 // per segment state: the particle order it was saved in
    int32_t *lam_id = nullptr, *lam_pos = nullptr;   // the adjoint state's order and an inverse-map scratch
    void *lam[2] = {nullptr, nullptr};
    mpm::AdjDev grid{};
    double *d_mubar[mpm::kMaxWalls] = {nullptr};
    void *final_S = nullptr;
    int32_t *final_id = nullptr, *final_sim = nullptr;
    bool allocated = false;
    // velocity monitors (Eulerian observations): boxes, steps, observed mean velocities
    int n_mon = 0, n_mobs = 0;
    std::vector<int> msteps;
    std::vector<double> mz;                    // n_mobs x n_mon x dim
    double *d_mboxes = nullptr, *d_msums = nullptr, *d_mg = nullptr;
    // after mpm_step_adjoint: lam[lam0] is the adjoint of the initial state, in order lam_id
    int lam0 = -1;
    // 3D single precision: scatter coefficients and, per sort generation of the segment
    // being reversed, its sort tables (tiles, count, position map, cell offsets)
    void *coef = nullptr;
    int gen_cap = 0;
    int4 *gen_tiles = nullptr;
    int32_t *gen_ntiles = nullptr, *gen_posmap = nullptr, *gen_celloff = nullptr;
    // the reverse sweep's stream and, per bank of kept states, the events that order
    // it against the recompute: bank filled (recomputed) and bank read (reversed)
    cudaStream_t rstream = nullptr;
    cudaEvent_t ev_filled[2] = {nullptr, nullptr}, ev_read[2] = {nullptr, nullptr};
};

// One saved copy of the particle state on the device.
struct StateSlot {
    void *S = nullptr;
    int32_t *id = nullptr, *sim = nullptr;
    int64_t n = 0;
};
constexpr int kMaxSlots = 16;

struct mpm_ctx {
    mpm_grid_desc grid{};
    mpm_material mat{};
    HostParams hp{};
    DevState ds{};
    const Ops *ops = nullptr;
    bool own_stream = false;
    bool need_sort = true;
    int64_t steps_since_sort = 0;
    int64_t steps = 0, sorts = 0, launches = 0;
    std::string err;
    // timing
    bool timing = false;
    std::vector<PendingTiming> pending;
    std::vector<cudaEvent_t> event_pool;
    double kt_ms[MPM_KERNEL_COUNT] = {0};
    int64_t kt_n[MPM_KERNEL_COUNT] = {0};
    int32_t *h_status = nullptr;       // pinned
    AdjHost adj;
    const AdjOps *aops = nullptr;
    StateSlot slots[kMaxSlots];
    int64_t adj_budget = 0;            // device bytes the adjoint may use to keep more than one segment
    double *diag_buf = nullptr;        // conservation sums (allocated by mpm_set_diagnostics)
    bool diag_valid = false;           // a step has run with the sums enabled
};

namespace {

int fail(mpm_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_fail(mpm_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, MPM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

bool forced_alloc_failure()
{
    const char *e = std::getenv("MPM_FAIL_ALLOC");
    return e && e[0] == '1';
}

template <class T> int dalloc(mpm_ctx *c, T **p, size_t count, const char *what)
{
    *p = nullptr;
    if (count == 0) count = 1;
    if (forced_alloc_failure()) return fail(c, MPM_ENOMEM, std::string("forced allocation failure: ") + what);
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, e == cudaErrorMemoryAllocation ? MPM_ENOMEM : MPM_ECUDA,
                    std::string("cudaMalloc ") + what + ": " + cudaGetErrorString(e));
    }
    return MPM_OK;
}

template <class T> void dfree(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

void free_adjoint(mpm_ctx *c)
{
    AdjHost &a = c->adj;
    dfree(a.d_ids); dfree(a.d_track_of_id); dfree(a.d_z); dfree(a.d_xobs);
    dfree(a.ckpt); dfree(a.seg); dfree(a.seg_grid); dfree(a.lam[0]); dfree(a.lam[1]);
    dfree(a.seg_id); dfree(a.lam_id); dfree(a.lam_pos);
    dfree(a.grid.GVB); dfree(a.grid.GAB);
    for (int w = 0; w < kMaxWalls; ++w) dfree(a.d_mubar[w]);
    dfree(a.final_S); dfree(a.final_id); dfree(a.final_sim);
    dfree(a.d_mboxes); dfree(a.d_msums); dfree(a.d_mg);
    dfree(a.coef); dfree(a.gen_tiles); dfree(a.gen_ntiles); dfree(a.gen_posmap); dfree(a.gen_celloff);
    for (int b = 0; b < 2; ++b) {
        if (a.ev_filled[b]) cudaEventDestroy(a.ev_filled[b]);
        if (a.ev_read[b]) cudaEventDestroy(a.ev_read[b]);
        a.ev_filled[b] = a.ev_read[b] = nullptr;
    }
    if (a.rstream) cudaStreamDestroy(a.rstream);
    a.rstream = nullptr;
    a.gen_cap = 0;
    a.ckpt_cap = a.seg_cap = 0;
    a.allocated = false;
    a.n_track = a.n_obs = 0;
    a.n_mon = a.n_mobs = 0;
    a.lam0 = -1;
}

void free_slots(mpm_ctx *c)
{
    for (auto &sl : c->slots) {
        dfree(sl.S);
        dfree(sl.id);
        dfree(sl.sim);
        sl.n = 0;
    }
}

void free_particles(mpm_ctx *c)
{
    free_adjoint(c);
    free_slots(c);
    DevState &d = c->ds;
    dfree(d.S); dfree(d.S2);
    dfree(d.id); dfree(d.id2); dfree(d.sim); dfree(d.sim2);
    dfree(d.keys[0]); dfree(d.keys[1]); dfree(d.vals[0]); dfree(d.vals[1]);
    dfree(d.hist); dfree(d.tiles); dfree(d.perm); dfree(d.posmap); dfree(d.cell_off); dfree(d.staging);
    c->hp.n = 0;
}

// Kernel timing brackets.
cudaEvent_t take_event(mpm_ctx *c)
{
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct TimingScope {
    mpm_ctx *c;
    int kernel;
    cudaStream_t stream;
    cudaEvent_t start = nullptr;
    TimingScope(mpm_ctx *c_, int k, cudaStream_t s = nullptr) : c(c_), kernel(k), stream(s ? s : c_->ds.stream)
    {
        if (c->timing) {
            start = take_event(c);
            cudaEventRecord(start, stream);
        }
    }
    ~TimingScope()
    {
        if (c->timing) {
            cudaEvent_t stop = take_event(c);
            cudaEventRecord(stop, stream);
            c->pending.push_back({kernel, start, stop});
        }
    }
};

void collect_timing(mpm_ctx *c)
{
    for (auto &p : c->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.stop) == cudaSuccess && cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
            c->kt_ms[p.kernel] += ms;
            c->kt_n[p.kernel] += 1;
        }
        c->event_pool.push_back(p.start);
        c->event_pool.push_back(p.stop);
    }
    c->pending.clear();
}

int check_launch(mpm_ctx *c, const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    return MPM_OK;
}

int do_sort(mpm_ctx *c)
{
    TimingScope ts(c, MPM_KERNEL_SORT);
    c->ops->keys(c->hp, c->ds);
    radix_sort_pairs(c->hp, c->ds);
    build_tiles(c->hp, c->ds);             // tile list, (rank, cell) order, gather permutation
    c->ops->permute(c->hp, c->ds);
    std::swap(c->ds.S, c->ds.S2);
    std::swap(c->ds.id, c->ds.id2);
    std::swap(c->ds.sim, c->ds.sim2);
    c->launches += 5 + 3 * ((c->ds.key_bits + kRadixBits - 1) / kRadixBits);
    c->sorts++;
    c->need_sort = false;
    c->steps_since_sort = 0;
    return check_launch(c, "sort");
}

int read_status(mpm_ctx *c)
{
    DevState &d = c->ds;
    cudaError_t e = cudaMemcpyAsync(c->h_status, d.status, sizeof(int32_t), cudaMemcpyDeviceToHost, d.stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "status read");
    e = cudaStreamSynchronize(d.stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    collect_timing(c);
    const int32_t s = *c->h_status;
    if (s & kStatusTimeout) return fail(c, MPM_ETIMEOUT, "a bounded device wait ran out (grid window copy)");
    if (s & kStatusNaN) return fail(c, MPM_ENAN, "a particle state became non-finite");
    if (s & kStatusChunkOverflow) return fail(c, MPM_ECUDA, "work chunk list overflow (internal)");
    return MPM_OK;
}

int field_width(const mpm_ctx *c, int field)
{
    const int d = c->grid.dim;
    switch (field) {
    case MPM_FIELD_X: case MPM_FIELD_V: return d;
    case MPM_FIELD_C: case MPM_FIELD_F: return d * d;
    case MPM_FIELD_RHO: case MPM_FIELD_EPS: return 1;
    case MPM_FIELD_SIGMA: return 9;
    default: return MPM_EINVAL;
    }
}

// TMA descriptor of the grid velocities V: dims (4 components, G_x, G_y, [G_z], batch),
// box (4, W, W, [W], 1) = the shared-memory window of one tile.
int make_tensor_map_V(mpm_ctx *c)
{
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || fn == nullptr || q != cudaDriverEntryPointSuccess)
        return fail(c, MPM_ECUDA, "cuTensorMapEncodeTiled is not available");
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const HostParams &h = c->hp;
    const int d = h.dim;
    const cuuint64_t rsz = h.precision == MPM_FP64 ? 8 : 4;
    cuuint64_t gdim[5], gstride[4];
    cuuint32_t box[5], estr[5];
    gdim[0] = 4;
    box[0] = 4;
    cuuint64_t stride = 4 * rsz;
    for (int a = 0; a < d; ++a) {
        gdim[1 + a] = (cuuint64_t)h.G_nodes[a];
        gstride[a] = stride;
        stride *= (cuuint64_t)h.G_nodes[a];
        box[1 + a] = (cuuint32_t)h.W;
    }
    gdim[d + 1] = (cuuint64_t)h.batch;
    gstride[d] = stride;
    box[d + 1] = 1;
    for (int i = 0; i < 5; ++i) estr[i] = 1;
    CUresult r = encode(&c->ds.tmap_V, rsz == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        (cuuint32_t)(d + 2), c->ds.V, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, MPM_ECUDA, "cuTensorMapEncodeTiled failed for the grid velocities");
    return MPM_OK;
}

}  // namespace

namespace {

// Positions outside [0, L] or not finite and simulation ids outside [0, batch):
// counted on the device for the device-pointer load.
__global__ void k_check_load(int64_t n, int d, const double *__restrict__ x, const int32_t *__restrict__ sim,
                             int batch, double L0, double L1, double L2, int32_t *__restrict__ bad)
{
    const double L[3] = {L0, L1, L2};
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        bool ok = true;
        for (int a = 0; a < d; ++a) {
            const double xa = x[p * d + a];
            ok = ok && (xa >= 0.0 && xa <= L[a]);
        }
        if (!ok) atomicOr(bad, 1);
        if (sim != nullptr && (sim[p] < 0 || sim[p] >= batch)) atomicOr(bad, 2);
    }
}

// mpm_load_particles and mpm_load_particles_dev: x, v, sim_id in host memory, or
// (device) in device memory read on the context's stream.
int load_particles(mpm_ctx *c, int64_t n, const double *x, const double *v, double particle_volume,
                   const int32_t *sim_id, bool device)
{
    const char *who = device ? "mpm_load_particles_dev" : "mpm_load_particles";
    if (!c || n <= 0 || !x || !(particle_volume > 0)) return fail(c, MPM_EINVAL, std::string(who) + ": bad argument");
    if (n > (int64_t)1 << 30) return fail(c, MPM_EINVAL, std::string(who) + ": too many particles");
    const int d = c->grid.dim;
    DevState &ds = c->ds;
    HostParams &h = c->hp;
    if (device) {                                  // the same checks, on the device
        int32_t *bad = nullptr;
        int rc = dalloc(c, &bad, 1, "load check");
        if (rc != MPM_OK) return rc;
        int32_t hbad = 0;
        cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int32_t), ds.stream);
        if (e == cudaSuccess) {
            const int nb = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ds.num_sms * 8);
            k_check_load<<<nb, 256, 0, ds.stream>>>(n, d, x, sim_id, c->grid.batch, h.n_cells[0] * h.dx,
                                                    h.n_cells[1] * h.dx, d == 3 ? h.n_cells[2] * h.dx : 0.0, bad);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, ds.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ds.stream);
        dfree(bad);
        if (e != cudaSuccess) return cuda_fail(c, e, "mpm_load_particles_dev: check");
        if (hbad & 1)
            return fail(c, MPM_EINVAL, "mpm_load_particles_dev: position outside the domain or not finite");
        if (hbad & 2) return fail(c, MPM_EINVAL, "mpm_load_particles_dev: simulation id out of range");
    } else {
        for (int64_t p = 0; p < n; ++p)
            for (int a = 0; a < d; ++a) {
                const double xa = x[p * d + a];
                if (!(xa >= 0.0 && xa <= c->hp.n_cells[a] * c->hp.dx))
                    return fail(c, MPM_EINVAL, "mpm_load_particles: position outside the domain or not finite");
            }
        if (sim_id)
            for (int64_t p = 0; p < n; ++p)
                if (sim_id[p] < 0 || sim_id[p] >= c->grid.batch)
                    return fail(c, MPM_EINVAL, "mpm_load_particles: simulation id out of range");
    }
    CK(cudaStreamSynchronize(ds.stream), "synchronize before load");
    free_particles(c);
    h.n = n;
    h.npad = (n + 63) / 64 * 64;                  // whole blocks of kPB particles
    h.vol0 = particle_volume;
    h.mass = h.rho0 * particle_volume;
    const size_t rsz = c->grid.precision == MPM_FP64 ? 8 : 4;
    const int nblk = (int)((n + kSortChunk - 1) / kSortChunk);
    {
        const int64_t all_tiles = (int64_t)c->grid.batch * h.tiles_per_sim;
        ds.max_tiles = all_tiles < n ? all_tiles : n;
    }
    const int TN = c->grid.dim == 2 ? Geo<2>::TN : Geo<3>::TN;
    int rc = MPM_OK;
    // 64 elements of slack: bulk copies of the last component may read up to 7 past npad
    if (rc == MPM_OK) rc = dalloc(c, (unsigned char **)&ds.S, ((size_t)h.ncomp * h.npad + 64) * rsz, "particle state");
    if (rc == MPM_OK)
        rc = dalloc(c, (unsigned char **)&ds.S2, ((size_t)h.ncomp * h.npad + 64) * rsz, "particle state (sort)");
    if (rc == MPM_OK) rc = dalloc(c, &ds.id, n, "ids");
    if (rc == MPM_OK) rc = dalloc(c, &ds.id2, n, "ids (sort)");
    if (rc == MPM_OK) rc = dalloc(c, &ds.sim, n, "sim ids");
    if (rc == MPM_OK) rc = dalloc(c, &ds.sim2, n, "sim ids (sort)");
    if (rc == MPM_OK) rc = dalloc(c, &ds.keys[0], n, "keys");
    if (rc == MPM_OK) rc = dalloc(c, &ds.keys[1], n, "keys");
    if (rc == MPM_OK) rc = dalloc(c, &ds.vals[0], n, "values");
    if (rc == MPM_OK) rc = dalloc(c, &ds.vals[1], n, "values");
    if (rc == MPM_OK) rc = dalloc(c, &ds.hist, (size_t)kRadixBins * nblk + kScanSegments, "histogram");
    if (rc == MPM_OK) rc = dalloc(c, &ds.tiles, 2 * ds.max_tiles, "tile list");     // key order + G2P order
    if (rc == MPM_OK) rc = dalloc(c, &ds.perm, n, "permutation");
    if (rc == MPM_OK) rc = dalloc(c, &ds.posmap, n, "position map");
    if (rc == MPM_OK) rc = dalloc(c, &ds.cell_off, (size_t)ds.max_tiles * (TN + 1), "cell offsets");
    if (rc == MPM_OK) rc = dalloc(c, &ds.staging, (size_t)n * 9, "staging");
    if (rc != MPM_OK) {
        free_particles(c);
        return rc;
    }
    const cudaMemcpyKind kind = device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(ds.staging, x, sizeof(double) * n * d, kind, ds.stream), "copy x");
    double *vdev = nullptr;
    if (v) {
        vdev = ds.staging + (size_t)n * d;
        CK(cudaMemcpyAsync(vdev, v, sizeof(double) * n * d, kind, ds.stream), "copy v");
    }
    if (sim_id) {
        CK(cudaMemcpyAsync(ds.sim, sim_id, sizeof(int32_t) * n, kind, ds.stream), "copy sim ids");
    } else {
        CK(cudaMemsetAsync(ds.sim, 0, sizeof(int32_t) * n, ds.stream), "zero sim ids");
    }
    c->ops->init_state(h, ds, ds.staging, vdev);
    c->launches++;
    CK(cudaGetLastError(), "init state");
    CK(cudaStreamSynchronize(ds.stream), "load particles");
    c->need_sort = true;
    return MPM_OK;
}

}  // namespace

namespace {

// The adjoint's device buffers, (re)allocated when too small: n_ckpt checkpoints,
// KS kept states with their grids and orders, gens generations of sort tables
// (3D single precision), the two adjoint states and grids, the final state.
int adj_buffers(mpm_ctx *c, int64_t n_ckpt, int64_t KS, int gens)
{
    AdjHost &a = c->adj;
    const HostParams &h = c->hp;
    DevState &ds = c->ds;
    const int NA = adj_ncomp_material(h.dim, c->mat.kind == MPM_DRUCKER_PRAGER ? 1 : 0);
    const size_t rsz = h.precision == MPM_FP64 ? 8 : 4;
    const int64_t n = h.n;
    const size_t st_bytes = (size_t)NA * n * rsz;
    const size_t gbytes = (size_t)h.nodes_per_sim * 4 * rsz;
    const size_t fbytes = ((size_t)(h.node_tiles_per_sim + 1) * sizeof(int32_t) + 255) / 256 * 256;
    const bool split = h.dim == 3 && h.precision == MPM_FP32;
    const int64_t TNc = 512 + 1;
    if (a.ckpt_cap < n_ckpt) {
        dfree(a.ckpt);
        int rc = dalloc(c, (unsigned char **)&a.ckpt, st_bytes * n_ckpt, "checkpoints");
        if (rc != MPM_OK) return rc;
        a.ckpt_cap = n_ckpt;
    }
    if (a.seg_cap < KS) {
        dfree(a.seg);
        dfree(a.seg_id);
        int rc = dalloc(c, (unsigned char **)&a.seg, st_bytes * KS, "segment states");
        if (rc == MPM_OK) rc = dalloc(c, &a.seg_id, (size_t)n * KS, "segment orders");
        if (rc != MPM_OK) return rc;
        a.seg_cap = KS;
    }
    if (a.seg_grid_cap < KS) {
        dfree(a.seg_grid);
        int rc = dalloc(c, (unsigned char **)&a.seg_grid, (2 * gbytes + fbytes) * KS, "segment grids");
        if (rc != MPM_OK) return rc;
        // nodes a step does not touch keep finite values from earlier steps (never read)
        CK(cudaMemsetAsync(a.seg_grid, 0, (2 * gbytes + fbytes) * KS, ds.stream), "zero segment grids");
        a.seg_grid_cap = KS;
    }
    if (split && a.gen_cap < gens) {
        dfree(a.coef); dfree(a.gen_tiles); dfree(a.gen_ntiles); dfree(a.gen_posmap); dfree(a.gen_celloff);
        int rc = dalloc(c, (unsigned char **)&a.coef, (size_t)21 * n * rsz, "scatter coefficients");
        if (rc == MPM_OK) rc = dalloc(c, &a.gen_tiles, (size_t)gens * ds.max_tiles, "generation tiles");
        if (rc == MPM_OK) rc = dalloc(c, &a.gen_ntiles, (size_t)gens, "generation tile counts");
        if (rc == MPM_OK) rc = dalloc(c, &a.gen_posmap, (size_t)gens * n, "generation position maps");
        if (rc == MPM_OK) rc = dalloc(c, &a.gen_celloff, (size_t)gens * ds.max_tiles * TNc, "generation offsets");
        if (rc != MPM_OK) return rc;
        a.gen_cap = gens;
    }
    if (!a.allocated) {
        // a failed earlier attempt may have left some of these allocated
        dfree(a.lam[0]); dfree(a.lam[1]); dfree(a.grid.GVB); dfree(a.grid.GAB);
        dfree(a.final_S); dfree(a.final_id); dfree(a.final_sim); dfree(a.lam_id); dfree(a.lam_pos);
        int rc = MPM_OK;
        if (rc == MPM_OK) rc = dalloc(c, (unsigned char **)&a.lam[0], st_bytes, "adjoint state");
        if (rc == MPM_OK) rc = dalloc(c, (unsigned char **)&a.lam[1], st_bytes, "adjoint state");
        if (rc == MPM_OK) rc = dalloc(c, (unsigned char **)&a.grid.GVB, gbytes, "adjoint grid");
        if (rc == MPM_OK) rc = dalloc(c, (unsigned char **)&a.grid.GAB, gbytes, "adjoint grid");
        if (rc == MPM_OK)
            rc = dalloc(c, (unsigned char **)&a.final_S, ((size_t)h.ncomp * h.npad + 64) * rsz, "final state");
        if (rc == MPM_OK) rc = dalloc(c, &a.final_id, n, "final ids");
        if (rc == MPM_OK) rc = dalloc(c, &a.final_sim, n, "final sims");
        if (rc == MPM_OK) rc = dalloc(c, &a.lam_id, n, "adjoint order");
        if (rc == MPM_OK) rc = dalloc(c, &a.lam_pos, n, "adjoint order");
        if (rc != MPM_OK) return rc;
        a.allocated = true;
    }
    return MPM_OK;
}

}  // namespace

extern "C" {

int mpm_create(const mpm_grid_desc *grid, const mpm_material *material, void *cuda_stream, mpm_ctx **out)
{
    if (!grid || !material || !out) return MPM_EINVAL;
    const mpm_grid_desc &g = *grid;
    const mpm_material &m = *material;
    if (g.dim != 2 && g.dim != 3) return MPM_EINVAL;
    for (int a = 0; a < g.dim; ++a)
        if (g.n_cells[a] < 1 || g.n_cells[a] > 4096) return MPM_EINVAL;
    if (!(g.dx > 0) || !(g.dt > 0) || g.sort_every < 1 || g.batch < 1) return MPM_EINVAL;
    if (!std::isfinite(g.dx) || !std::isfinite(g.dt)) return MPM_EINVAL;
    for (int a = 0; a < g.dim; ++a)
        if (!std::isfinite(g.gravity[a])) return MPM_EINVAL;
    if (g.transfer < MPM_TRANSFER_APIC || g.transfer > MPM_TRANSFER_FLIP) return MPM_EINVAL;
    if (g.transfer == MPM_TRANSFER_FLIP && !(g.flip_alpha >= 0.0 && g.flip_alpha <= 1.0)) return MPM_EINVAL;
    if (g.precision != MPM_FP32 && g.precision != MPM_FP64) return MPM_EINVAL;
    if (m.kind != MPM_FLUID && m.kind != MPM_DRUCKER_PRAGER) return MPM_EINVAL;
    if (!(m.rho0 > 0) || !std::isfinite(m.rho0)) return MPM_EINVAL;
    if (m.kind == MPM_FLUID && (!(m.bulk_K > 0) || !(m.gamma > 0) || m.viscosity != 0.0 ||
                                !std::isfinite(m.bulk_K) || !std::isfinite(m.gamma)))
        return MPM_EINVAL;
    if (m.kind == MPM_DRUCKER_PRAGER &&
        (!(m.E > 0) || !std::isfinite(m.E) || !(m.nu > -1.0 && m.nu < 0.5) || !(m.phi_deg >= 0.0 && m.phi_deg < 90.0) ||
         !(m.psi_deg >= 0.0 && m.psi_deg < 90.0) || !(m.cohesion >= 0.0) || !std::isfinite(m.cohesion) ||
         !(m.sigma_t >= 0.0) || !std::isfinite(m.sigma_t)))
        return MPM_EINVAL;

    mpm_ctx *c = new mpm_ctx();
    c->grid = g;
    c->mat = m;
    HostParams &h = c->hp;
    h.dim = g.dim;
    h.batch = g.batch;
    h.transfer = g.transfer;
    h.flip_alpha = g.flip_alpha;
    h.precision = g.precision;
    h.material = m.kind;
    h.dp_literal = m.dp_literal ? 1 : 0;
    h.dx = g.dx;
    h.dt = g.dt;
    for (int a = 0; a < 3; ++a) {
        h.n_cells[a] = a < g.dim ? g.n_cells[a] : 1;
        h.gravity[a] = a < g.dim ? g.gravity[a] : 0.0;
    }
    h.rho0 = m.rho0;
    h.bulk_K = m.bulk_K;
    h.gamma = m.gamma;
    h.m_eps = 1e-10 * m.rho0 * std::pow(g.dx, g.dim);
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
    const int T = g.dim == 2 ? Geo<2>::T : Geo<3>::T;
    h.T = T;
    h.W = T + 4;
    h.nodes_per_sim = 1;
    h.tiles_per_sim = 1;
    h.node_tiles_per_sim = 1;
    for (int a = 0; a < 3; ++a) {
        if (a < g.dim) {
            h.n_tiles[a] = h.n_cells[a] / T + 1;
            h.G_nodes[a] = h.n_tiles[a] * T + 4;
            h.node_tiles[a] = (h.G_nodes[a] + T - 1) / T;
        } else {
            h.n_tiles[a] = h.G_nodes[a] = h.node_tiles[a] = 1;
        }
        h.nodes_per_sim *= h.G_nodes[a];
        h.tiles_per_sim *= h.n_tiles[a];
        h.node_tiles_per_sim *= h.node_tiles[a];
    }
    const int cell_bits = g.dim == 2 ? Geo<2>::CELL_BITS : Geo<3>::CELL_BITS;
    int tbits = 0;
    while ((int64_t(1) << tbits) < (int64_t)g.batch * h.tiles_per_sim) ++tbits;
    c->ds.key_bits = tbits + cell_bits;
    if (c->ds.key_bits > 32) {
        delete c;
        return MPM_EINVAL;
    }
    const int d = g.dim;
    // component order: what G2P reads (x, F, rho [, sigma, eps]) first, then v, C
    h.off_x = 0;
    h.off_F = d;
    h.off_rho = d + d * d;
    h.off_sig = h.off_rho + 1;
    h.off_eps = h.off_sig + 6;
    h.off_v = m.kind == MPM_DRUCKER_PRAGER ? h.off_eps + 1 : h.off_rho + 1;
    h.off_C = h.off_v + d;
    h.ncomp = h.off_C + d * d;
    c->ops = g.precision == MPM_FP64 ? &ops_f64 : &ops_f32;
    c->aops = g.precision == MPM_FP64 ? &adj_ops_f64 : &adj_ops_f32;

    DevState &ds = c->ds;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ds.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete c;
        return MPM_ECUDA;
    }
    if (cuda_stream) {
        ds.stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ds.stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return MPM_ECUDA;
        }
        c->own_stream = true;
    }
    const size_t rsz = g.precision == MPM_FP64 ? 8 : 4;
    const int64_t nodes = (int64_t)g.batch * h.nodes_per_sim;
    const int64_t ntiles = (int64_t)g.batch * h.tiles_per_sim;
    int rc = MPM_OK;
    if (rc == MPM_OK) rc = dalloc(c, (unsigned char **)&ds.A, nodes * 4 * rsz, "grid accumulators");
    if (rc == MPM_OK) rc = dalloc(c, (unsigned char **)&ds.V, nodes * 4 * rsz, "grid velocities");
    if (rc == MPM_OK && g.transfer == MPM_TRANSFER_FLIP) {
        rc = dalloc(c, (unsigned char **)&ds.A2, nodes * 4 * rsz, "FLIP grid momenta");
        if (rc == MPM_OK) rc = dalloc(c, (unsigned char **)&ds.V2, nodes * 4 * rsz, "FLIP grid velocities");
        if (rc == MPM_OK) cudaMemsetAsync(ds.A2, 0, nodes * 4 * rsz, ds.stream);
        if (rc == MPM_OK) cudaMemsetAsync(ds.V2, 0, nodes * 4 * rsz, ds.stream);
    }
    if (rc == MPM_OK) rc = dalloc(c, &ds.flags, (size_t)g.batch * h.node_tiles_per_sim, "node tile flags");
    if (rc == MPM_OK) rc = dalloc(c, &ds.tile_start, ntiles, "tile starts");
    if (rc == MPM_OK) rc = dalloc(c, &ds.tile_end, ntiles, "tile ends");
    if (rc == MPM_OK) rc = dalloc(c, &ds.counters, 8, "counters");
    if (rc == MPM_OK) rc = dalloc(c, &ds.node_list, (size_t)g.batch * h.node_tiles_per_sim, "node tile list");
    if (rc == MPM_OK) rc = dalloc(c, &ds.status, 1, "status");
    if (rc == MPM_OK) rc = dalloc(c, &ds.escaped, 1, "escape counter");
    if (rc == MPM_OK && cudaMallocHost((void **)&c->h_status, sizeof(int32_t)) != cudaSuccess) rc = MPM_ENOMEM;
    if (rc == MPM_OK) {
        cudaMemsetAsync(ds.A, 0, nodes * 4 * rsz, ds.stream);
        cudaMemsetAsync(ds.V, 0, nodes * 4 * rsz, ds.stream);
        cudaMemsetAsync(ds.flags, 0, sizeof(uint32_t) * g.batch * h.node_tiles_per_sim, ds.stream);
        cudaMemsetAsync(ds.counters, 0, sizeof(int32_t) * 8, ds.stream);
        cudaMemsetAsync(ds.status, 0, sizeof(int32_t), ds.stream);
        cudaMemsetAsync(ds.escaped, 0, sizeof(unsigned long long), ds.stream);
        if (cudaStreamSynchronize(ds.stream) != cudaSuccess) rc = MPM_ECUDA;
    }
    if (rc == MPM_OK) rc = make_tensor_map_V(c);
    if (rc != MPM_OK) {
        mpm_destroy(c);
        return rc;
    }
    *out = c;
    return MPM_OK;
}

void mpm_destroy(mpm_ctx *c)
{
    if (!c) return;
    DevState &d = c->ds;
    if (d.stream) cudaStreamSynchronize(d.stream);
    collect_timing(c);
    free_particles(c);
    dfree(d.A); dfree(d.V); dfree(d.A2); dfree(d.V2); dfree(d.flags); dfree(d.node_list);
    dfree(d.tile_start); dfree(d.tile_end);
    dfree(d.counters); dfree(d.status); dfree(d.escaped); dfree(c->diag_buf);
    for (int w = 0; w < kMaxWalls; ++w) dfree(d.mu_dev[w]);
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->own_stream && d.stream) cudaStreamDestroy(d.stream);
    delete c;
}

int mpm_load_particles(mpm_ctx *c, int64_t n, const double *x, const double *v, double particle_volume,
                       const int32_t *sim_id)
{
    return load_particles(c, n, x, v, particle_volume, sim_id, false);
}

int mpm_load_particles_dev(mpm_ctx *c, int64_t n, const double *x_dev, const double *v_dev, double particle_volume,
                           const int32_t *sim_id_dev)
{
    return load_particles(c, n, x_dev, v_dev, particle_volume, sim_id_dev, true);
}

int mpm_set_particle_field(mpm_ctx *c, int field, const double *values)
{
    if (!c || !values) return fail(c, MPM_EINVAL, "mpm_set_particle_field: bad argument");
    if (c->hp.n == 0) return fail(c, MPM_ESTATE, "mpm_set_particle_field: no particles loaded");
    const int wdt = field_width(c, field);
    if (wdt < 0) return fail(c, MPM_EINVAL, "mpm_set_particle_field: unknown field");
    if (field == MPM_FIELD_SIGMA && c->mat.kind != MPM_DRUCKER_PRAGER)
        return fail(c, MPM_EINVAL, "mpm_set_particle_field: fluid stress follows from the density");
    if (field == MPM_FIELD_EPS && c->mat.kind != MPM_DRUCKER_PRAGER)
        return fail(c, MPM_EINVAL, "mpm_set_particle_field: no plastic strain in a fluid");
    if (field == MPM_FIELD_X) {
        const int d = c->grid.dim;
        for (int64_t p = 0; p < c->hp.n; ++p)
            for (int a = 0; a < d; ++a) {
                const double xa = values[p * d + a];
                if (!(xa >= 0.0 && xa <= c->hp.n_cells[a] * c->hp.dx))
                    return fail(c, MPM_EINVAL, "mpm_set_particle_field: position outside the domain or not finite");
            }
    }
    DevState &ds = c->ds;
    CK(cudaMemcpyAsync(ds.staging, values, sizeof(double) * c->hp.n * wdt, cudaMemcpyHostToDevice, ds.stream),
       "copy field");
    c->ops->set_field(c->hp, ds, field, ds.staging);
    c->launches++;
    CK(cudaGetLastError(), "set field");
    CK(cudaStreamSynchronize(ds.stream), "set field");
    if (field == MPM_FIELD_X) c->need_sort = true;
    return MPM_OK;
}

int mpm_set_friction_field(mpm_ctx *c, int wall, const int n_seg[2], const double *mu)
{
    if (!c || !n_seg || !mu) return fail(c, MPM_EINVAL, "mpm_set_friction_field: bad argument");
    if (wall < 0 || wall >= 2 * c->grid.dim) return fail(c, MPM_EINVAL, "mpm_set_friction_field: bad wall");
    const int ns1 = c->grid.dim == 2 ? 1 : n_seg[1];
    if (n_seg[0] < 1 || ns1 < 1 || n_seg[0] > 65536 || ns1 > 65536)
        return fail(c, MPM_EINVAL, "mpm_set_friction_field: bad segment count");
    const int64_t count = (int64_t)c->grid.batch * n_seg[0] * ns1;
    for (int64_t i = 0; i < count; ++i)
        if (!(mu[i] >= 0.0)) return fail(c, MPM_EINVAL, "mpm_set_friction_field: negative or non-finite mu");
    DevState &ds = c->ds;
    CK(cudaStreamSynchronize(ds.stream), "synchronize before friction update");
    dfree(ds.mu_dev[wall]);
    const size_t rsz = c->grid.precision == MPM_FP64 ? 8 : 4;
    unsigned char *buf = nullptr;
    int rc = dalloc(c, &buf, (size_t)count * rsz, "friction field");
    if (rc != MPM_OK) return rc;
    if (c->grid.precision == MPM_FP64) {
        CK(cudaMemcpy(buf, mu, sizeof(double) * count, cudaMemcpyHostToDevice), "copy friction");
    } else {
        std::vector<float> tmp(count);
        for (int64_t i = 0; i < count; ++i) tmp[i] = (float)mu[i];
        CK(cudaMemcpy(buf, tmp.data(), sizeof(float) * count, cudaMemcpyHostToDevice), "copy friction");
    }
    ds.mu_dev[wall] = buf;
    ds.n_seg[wall][0] = n_seg[0];
    ds.n_seg[wall][1] = ns1;
    return MPM_OK;
}

int mpm_set_obstacles(mpm_ctx *c, int n_obstacles, const double *boxes)
{
    if (!c || n_obstacles < 0 || n_obstacles > MPM_MAX_OBSTACLES || (n_obstacles > 0 && !boxes))
        return fail(c, MPM_EINVAL, "mpm_set_obstacles: bad argument");
    const int d = c->grid.dim;
    Obstacles ob{};
    ob.n = n_obstacles;
    for (int o = 0; o < n_obstacles; ++o) {
        const double *lo = boxes + (size_t)o * 2 * d, *hi = lo + d;
        int faces = 0;
        for (int a = 0; a < d; ++a) {
            if (!(lo[a] <= hi[a]) || !std::isfinite(lo[a]) || !std::isfinite(hi[a]))
                return fail(c, MPM_EINVAL, "mpm_set_obstacles: bad box");
            // node extents of the closed box (1e-9 dx tolerance), clamped to the node range
            const double l = std::ceil(lo[a] / c->grid.dx - 1e-9), u = std::floor(hi[a] / c->grid.dx + 1e-9);
            const double big = c->grid.n_cells[a] + 8.0;
            ob.lo[o][a] = (int)std::max(-8.0, std::min(big, l));
            ob.hi[o][a] = (int)std::max(-8.0, std::min(big, u));
            if (l > 0.0) faces |= 1 << (2 * a);
            if (u < c->grid.n_cells[a]) faces |= 1 << (2 * a + 1);
        }
        if (faces == 0) return fail(c, MPM_EINVAL, "mpm_set_obstacles: box has no face inside the domain");
        ob.faces[o] = faces;
    }
    CK(cudaStreamSynchronize(c->ds.stream), "synchronize before obstacle update");
    c->hp.obs = ob;
    return MPM_OK;
}

}  // extern "C"

namespace {
int step_many(mpm_ctx *c, int n_steps)
{
    for (int s = 0; s < n_steps; ++s) {
        if (c->need_sort || c->steps_since_sort >= c->grid.sort_every) {
            int rc = do_sort(c);
            if (rc != MPM_OK) return rc;
        }
        if (c->ds.diag != nullptr) {           // conservation sums of this step: cleared, then the particles
            CK(cudaMemsetAsync(c->ds.diag, 0, sizeof(double) * kDiagCount, c->ds.stream), "diagnostics clear");
            c->ops->diag_particles(c->hp, c->ds);
            c->launches++;
            c->diag_valid = true;
        }
        {
            TimingScope ts(c, MPM_KERNEL_P2G);
            c->ops->p2g(c->hp, c->ds);
        }
        {
            TimingScope ts(c, MPM_KERNEL_GRID);
            c->ops->grid(c->hp, c->ds);
        }
        {
            TimingScope ts(c, MPM_KERNEL_G2P);
            c->ops->g2p(c->hp, c->ds);
        }
        c->launches += 3;
        int rc = check_launch(c, "mpm_step");
        if (rc != MPM_OK) return rc;
        c->steps_since_sort++;
        c->steps++;
    }
    return MPM_OK;
}
}  // namespace

extern "C" {

int mpm_step(mpm_ctx *c, int n_steps)
{
    if (!c || n_steps < 0) return fail(c, MPM_EINVAL, "mpm_step: bad argument");
    if (c->hp.n == 0) return fail(c, MPM_ESTATE, "mpm_step: no particles loaded");
    return step_many(c, n_steps);
}

int mpm_request_sort(mpm_ctx *c)
{
    if (!c) return MPM_EINVAL;
    c->need_sort = true;
    return MPM_OK;
}

int mpm_set_diagnostics(mpm_ctx *c, int enable)
{
    if (!c) return MPM_EINVAL;
    if (enable) {
        if (c->diag_buf == nullptr) {
            int rc = dalloc(c, &c->diag_buf, kDiagCount, "diagnostics");
            if (rc != MPM_OK) return rc;
            CK(cudaMemsetAsync(c->diag_buf, 0, sizeof(double) * kDiagCount, c->ds.stream), "diagnostics clear");
        }
        c->ds.diag = c->diag_buf;
    } else {
        c->ds.diag = nullptr;
    }
    return MPM_OK;
}

int mpm_get_diagnostics(mpm_ctx *c, double *out, int n)
{
    if (!c || !out || n < 0) return fail(c, MPM_EINVAL, "mpm_get_diagnostics: bad argument");
    if (!c->diag_valid || c->diag_buf == nullptr)
        return fail(c, MPM_ESTATE, "mpm_get_diagnostics: no step has run with the diagnostics enabled");
    double h[kDiagCount];
    CK(cudaMemcpyAsync(h, c->diag_buf, sizeof(h), cudaMemcpyDeviceToHost, c->ds.stream), "diagnostics read");
    CK(cudaStreamSynchronize(c->ds.stream), "diagnostics read");
    for (int i = 0; i < n && i < kDiagCount; ++i) out[i] = h[i];
    return MPM_OK;
}

int mpm_set_debug(mpm_ctx *c, int flags)
{
    if (!c || (flags & ~kDebugWithholdWindowCopy) != 0) return fail(c, MPM_EINVAL, "mpm_set_debug: unknown flag");
    c->hp.debug = flags;
    return MPM_OK;
}

int mpm_synchronize(mpm_ctx *c)
{
    if (!c) return MPM_EINVAL;
    return read_status(c);
}

int mpm_get_particles(mpm_ctx *c, int field, double *out)
{
    if (!c || !out) return fail(c, MPM_EINVAL, "mpm_get_particles: bad argument");
    if (c->hp.n == 0) return fail(c, MPM_ESTATE, "mpm_get_particles: no particles loaded");
    const int wdt = field_width(c, field);
    if (wdt < 0) return fail(c, MPM_EINVAL, "mpm_get_particles: unknown field");
    DevState &ds = c->ds;
    c->ops->get_field(c->hp, ds, field, ds.staging);
    c->launches++;
    CK(cudaGetLastError(), "get field");
    CK(cudaMemcpyAsync(out, ds.staging, sizeof(double) * c->hp.n * wdt, cudaMemcpyDeviceToHost, ds.stream),
       "copy field to host");
    return read_status(c);
}

int mpm_get_particles_dev(mpm_ctx *c, int field, double *out_dev)
{
    if (!c || !out_dev) return fail(c, MPM_EINVAL, "mpm_get_particles_dev: bad argument");
    if (c->hp.n == 0) return fail(c, MPM_ESTATE, "mpm_get_particles_dev: no particles loaded");
    if (field_width(c, field) < 0) return fail(c, MPM_EINVAL, "mpm_get_particles_dev: unknown field");
    c->ops->get_field(c->hp, c->ds, field, out_dev);      // written on the context's stream, no wait
    c->launches++;
    CK(cudaGetLastError(), "get field");
    return MPM_OK;
}

int mpm_field_width(const mpm_ctx *c, int field)
{
    if (!c) return MPM_EINVAL;
    return field_width(c, field);
}

int64_t mpm_num_particles(const mpm_ctx *c) { return c ? c->hp.n : 0; }

int mpm_last_error(const mpm_ctx *c, char *buf, int len)
{
    if (!c || !buf || len <= 0) return MPM_EINVAL;
    std::snprintf(buf, (size_t)len, "%s", c->err.c_str());
    return MPM_OK;
}

int mpm_set_timing(mpm_ctx *c, int enable)
{
    if (!c) return MPM_EINVAL;
    c->timing = enable != 0;
    return MPM_OK;
}

int mpm_get_timing(mpm_ctx *c, int kernel, double *total_ms, int64_t *launches)
{
    if (!c || kernel < 0 || kernel >= MPM_KERNEL_COUNT || !total_ms || !launches) return MPM_EINVAL;
    CK(cudaStreamSynchronize(c->ds.stream), "timing synchronize");
    collect_timing(c);
    *total_ms = c->kt_ms[kernel];
    *launches = c->kt_n[kernel];
    return MPM_OK;
}

int mpm_reset_timing(mpm_ctx *c)
{
    if (!c) return MPM_EINVAL;
    CK(cudaStreamSynchronize(c->ds.stream), "timing synchronize");
    collect_timing(c);
    for (int k = 0; k < MPM_KERNEL_COUNT; ++k) {
        c->kt_ms[k] = 0.0;
        c->kt_n[k] = 0;
    }
    return MPM_OK;
}

int mpm_get_stats(mpm_ctx *c, int64_t *out, int n)
{
    if (!c || !out || n < 0) return MPM_EINVAL;
    int32_t cnt[2] = {0, 0};
    unsigned long long esc = 0;
    CK(cudaMemcpyAsync(cnt, c->ds.counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->ds.stream), "stats");
    CK(cudaMemcpyAsync(&esc, c->ds.escaped, sizeof(esc), cudaMemcpyDeviceToHost, c->ds.stream), "stats");
    CK(cudaStreamSynchronize(c->ds.stream), "stats");
    const int64_t vals[6] = {cnt[1], cnt[1], (int64_t)esc, c->sorts, c->steps, c->launches};
    for (int i = 0; i < n && i < 6; ++i) out[i] = vals[i];
    return MPM_OK;
}

int mpm_set_observations(mpm_ctx *c, int n_track, const int64_t *ids, int n_obs, const int *steps,
                         const double *z_obs)
{
    if (c && n_track == 0) {                      // clear the tracked-particle observations
        c->adj.n_track = c->adj.n_obs = 0;
        return MPM_OK;
    }
    if (!c || n_track < 0 || n_obs <= 0 || !ids || !steps || !z_obs)
        return fail(c, MPM_EINVAL, "mpm_set_observations: bad argument");
    const int64_t n = c->hp.n;
    if (n == 0) return fail(c, MPM_ESTATE, "mpm_set_observations: no particles loaded");
    std::vector<int32_t> track_of_id(n, -1);
    for (int l = 0; l < n_track; ++l) {
        if (ids[l] < 0 || ids[l] >= n) return fail(c, MPM_EINVAL, "mpm_set_observations: id out of range");
        if (track_of_id[ids[l]] >= 0) return fail(c, MPM_EINVAL, "mpm_set_observations: repeated id");
        track_of_id[ids[l]] = l;
    }
    for (int o = 0; o < n_obs; ++o)
        if (steps[o] < 1 || (o > 0 && steps[o] <= steps[o - 1]))
            return fail(c, MPM_EINVAL, "mpm_set_observations: steps must be >= 1 and increasing");
    AdjHost &a = c->adj;
    dfree(a.d_ids); dfree(a.d_track_of_id); dfree(a.d_z); dfree(a.d_xobs);
    const int d = c->grid.dim;
    int rc = MPM_OK;
    if (rc == MPM_OK) rc = dalloc(c, &a.d_ids, n_track, "tracked ids");
    if (rc == MPM_OK) rc = dalloc(c, &a.d_track_of_id, n, "track map");
    if (rc == MPM_OK) rc = dalloc(c, &a.d_z, (size_t)n_obs * n_track * d, "observations");
    if (rc == MPM_OK) rc = dalloc(c, &a.d_xobs, (size_t)n_obs * n_track * d, "observed positions");
    if (rc != MPM_OK) return rc;
    CK(cudaMemcpy(a.d_ids, ids, sizeof(int64_t) * n_track, cudaMemcpyHostToDevice), "copy ids");
    CK(cudaMemcpy(a.d_track_of_id, track_of_id.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice), "copy map");
    CK(cudaMemcpy(a.d_z, z_obs, sizeof(double) * n_obs * n_track * d, cudaMemcpyHostToDevice), "copy z");
    a.n_track = n_track;
    a.n_obs = n_obs;
    a.ids.assign(ids, ids + n_track);
    a.steps.assign(steps, steps + n_obs);
    a.z.assign(z_obs, z_obs + (size_t)n_obs * n_track * d);
    return MPM_OK;
}

int mpm_set_velocity_monitors(mpm_ctx *c, int n_mon, const double *boxes, int n_obs, const int *steps,
                              const double *v_obs)
{
    if (c && n_mon == 0) {                        // clear the monitors
        c->adj.n_mon = c->adj.n_mobs = 0;
        return MPM_OK;
    }
    if (!c || n_mon < 0 || n_mon > kMaxMonitors || n_obs <= 0 || !boxes || !steps || !v_obs)
        return fail(c, MPM_EINVAL, "mpm_set_velocity_monitors: bad argument");
    const int d = c->grid.dim;
    for (int l = 0; l < n_mon; ++l)
        for (int a = 0; a < d; ++a) {
            const double lo = boxes[(size_t)l * 2 * d + a], hi = boxes[(size_t)l * 2 * d + d + a];
            if (!(lo <= hi) || !std::isfinite(lo) || !std::isfinite(hi))
                return fail(c, MPM_EINVAL, "mpm_set_velocity_monitors: bad box");
        }
    for (int o = 0; o < n_obs; ++o)
        if (steps[o] < 1 || (o > 0 && steps[o] <= steps[o - 1]))
            return fail(c, MPM_EINVAL, "mpm_set_velocity_monitors: steps must be >= 1 and increasing");
    AdjHost &a = c->adj;
    dfree(a.d_mboxes); dfree(a.d_msums); dfree(a.d_mg);
    int rc = dalloc(c, &a.d_mboxes, (size_t)n_mon * 2 * d, "monitor boxes");
    if (rc == MPM_OK) rc = dalloc(c, &a.d_msums, (size_t)n_obs * n_mon * (d + 1), "monitor sums");
    if (rc == MPM_OK) rc = dalloc(c, &a.d_mg, (size_t)n_obs * n_mon * d, "monitor seeds");
    if (rc != MPM_OK) return rc;
    CK(cudaMemcpy(a.d_mboxes, boxes, sizeof(double) * n_mon * 2 * d, cudaMemcpyHostToDevice), "copy boxes");
    a.n_mon = n_mon;
    a.n_mobs = n_obs;
    a.msteps.assign(steps, steps + n_obs);
    a.mz.assign(v_obs, v_obs + (size_t)n_obs * n_mon * d);
    return MPM_OK;
}

int mpm_monitor_means(mpm_ctx *c, int n_mon, const double *boxes, double *out)
{
    if (!c || n_mon < 1 || n_mon > kMaxMonitors || !boxes || !out)
        return fail(c, MPM_EINVAL, "mpm_monitor_means: bad argument");
    if (c->hp.n == 0) return fail(c, MPM_ESTATE, "mpm_monitor_means: no particles loaded");
    if (c->grid.batch != 1) return fail(c, MPM_EINVAL, "mpm_monitor_means: batch must be 1");
    const HostParams &h = c->hp;
    DevState &ds = c->ds;
    const int d = h.dim;
    for (int l = 0; l < n_mon; ++l)
        for (int a = 0; a < d; ++a) {
            const double lo = boxes[(size_t)l * 2 * d + a], hi = boxes[(size_t)l * 2 * d + d + a];
            if (!(lo <= hi) || !std::isfinite(lo) || !std::isfinite(hi))
                return fail(c, MPM_EINVAL, "mpm_monitor_means: bad box");
        }
    double *dev = nullptr;
    int rc = dalloc(c, &dev, (size_t)n_mon * (3 * d + 1), "monitor scratch");
    if (rc != MPM_OK) return rc;
    double *dboxes = dev + (size_t)n_mon * (d + 1);
    cudaError_t e = cudaMemcpyAsync(dboxes, boxes, sizeof(double) * n_mon * 2 * d, cudaMemcpyHostToDevice, ds.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev, 0, sizeof(double) * n_mon * (d + 1), ds.stream);
    if (e == cudaSuccess) {
        const size_t rsz = h.precision == MPM_FP64 ? 8 : 4, rs = rsz * (size_t)kPB;
        c->aops->monitor_sum(h, ds, (char *)ds.S + rs * h.off_x, (char *)ds.S + rs * h.off_v, -h.ncomp, n_mon, dboxes,
                             dev);
        e = cudaMemcpyAsync(out, dev, sizeof(double) * n_mon * (d + 1), cudaMemcpyDeviceToHost, ds.stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ds.stream);
    dfree(dev);
    if (e != cudaSuccess) return fail(c, MPM_ECUDA, "mpm_monitor_means: device error");
    for (int l = 0; l < n_mon; ++l) {
        double *o = out + (size_t)l * (d + 1);
        if (o[d] > 0.0)
            for (int a = 0; a < d; ++a) o[a] /= o[d];
    }
    return MPM_OK;
}

int mpm_set_adjoint_memory(mpm_ctx *c, int64_t bytes)
{
    if (!c || bytes < 0) return fail(c, MPM_EINVAL, "mpm_set_adjoint_memory: bad argument");
    c->adj_budget = bytes;
    return MPM_OK;
}

int mpm_adjoint_width(const mpm_ctx *c)
{
    if (!c) return MPM_EINVAL;
    return adj_ncomp_material(c->grid.dim, c->mat.kind == MPM_DRUCKER_PRAGER ? 1 : 0);
}

int mpm_step_adjoint_1(mpm_ctx *c, int wall, const double *lam_next, double *lam_prev, double *dL_dmu_out)
{
    if (!c || !lam_next || !lam_prev || (wall >= 0 && !dL_dmu_out))
        return fail(c, MPM_EINVAL, "mpm_step_adjoint_1: bad argument");
    if (c->hp.n == 0) return fail(c, MPM_ESTATE, "mpm_step_adjoint_1: no particles loaded");
    if (c->grid.batch != 1) return fail(c, MPM_EINVAL, "mpm_step_adjoint_1: batch must be 1");
    if (c->grid.transfer != MPM_TRANSFER_APIC)
        return fail(c, MPM_EINVAL, "mpm_step_adjoint_1: the adjoint follows the APIC transfer");
    if (wall < -1 || wall >= 2 * c->grid.dim || (wall >= 0 && c->ds.mu_dev[wall] == nullptr))
        return fail(c, MPM_EINVAL, "mpm_step_adjoint_1: the wall has no friction field");
    AdjHost &a = c->adj;
    a.lam0 = -1;
    const HostParams &h = c->hp;
    DevState &ds = c->ds;
    const int d = h.dim;
    const int NA = adj_ncomp_material(d, c->mat.kind == MPM_DRUCKER_PRAGER ? 1 : 0);
    const size_t rsz = h.precision == MPM_FP64 ? 8 : 4;
    const int64_t n = h.n;
    const size_t gbytes = (size_t)h.nodes_per_sim * 4 * rsz;
    const bool split = d == 3 && h.precision == MPM_FP32;
    const int64_t TNc = 512 + 1;
    // one kept state with its grids and, for the cell-ordered v_bar scatter, one
    // generation of sort tables (the buffers of mpm_step_adjoint, at least one slot)
    int rc = adj_buffers(c, 0, 1, split ? 1 : 0);
    if (rc != MPM_OK) return rc;
    MuBar mub{};
    if (wall >= 0) {
        const int64_t cnt = (int64_t)ds.n_seg[wall][0] * ds.n_seg[wall][1];
        if (a.d_mubar[wall] == nullptr) {
            rc = dalloc(c, &a.d_mubar[wall], cnt, "dL/dmu");
            if (rc != MPM_OK) return rc;
        }
        CK(cudaMemsetAsync(a.d_mubar[wall], 0, sizeof(double) * cnt, ds.stream), "zero dL/dmu");
        mub.w[wall] = a.d_mubar[wall];
    }
    double *io = nullptr;                          // lam_next in, lam_prev out (load order, doubles)
    rc = dalloc(c, &io, (size_t)n * NA, "adjoint transfer");
    if (rc != MPM_OK) return rc;
    auto done = [&](int r) {
        dfree(io);
        return r;
    };
    // the step S^t -> S^{t+1}, keeping S^t, its grids and its sort tables
    if (c->need_sort || c->steps_since_sort >= c->grid.sort_every) {
        rc = do_sort(c);
        if (rc != MPM_OK) return done(rc);
    }
    int32_t *order = a.seg_id;                     // the order of S^t (and of S^{t+1})
    cudaError_t e = cudaMemcpyAsync(order, ds.id, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ds.stream);
    AdjDev ad = a.grid;
    if (e == cudaSuccess && split) {
        e = cudaMemcpyAsync(a.gen_tiles, ds.tiles, sizeof(int4) * ds.max_tiles, cudaMemcpyDeviceToDevice, ds.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(a.gen_ntiles, ds.counters + 1, sizeof(int32_t), cudaMemcpyDeviceToDevice, ds.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(a.gen_posmap, ds.posmap, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ds.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(a.gen_celloff, ds.cell_off, sizeof(int32_t) * ds.max_tiles * TNc,
                                cudaMemcpyDeviceToDevice, ds.stream);
        ad.coef = a.coef;
        ad.cursor = ds.counters + 5;
        ad.tiles = a.gen_tiles;
        ad.n_tiles = a.gen_ntiles;
        ad.posmap = a.gen_posmap;
        ad.cell_off = a.gen_celloff;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(a.grid.GVB, 0, gbytes, ds.stream);
    if (e != cudaSuccess) return done(cuda_fail(c, e, "mpm_step_adjoint_1: keep"));
    void *st = a.seg;
    void *GA = a.seg_grid, *GV = (char *)a.seg_grid + gbytes;
    int32_t *GL = (int32_t *)((char *)a.seg_grid + 2 * gbytes);
    ds.save_S = st;
    ds.save_A = GA;
    ds.save_V = GV;
    ds.save_L = GL;
    rc = step_many(c, 1);
    ds.save_S = ds.save_A = ds.save_V = nullptr;
    ds.save_L = nullptr;
    if (rc != MPM_OK) return done(rc);
    // the reverse step: lam_next in the particle order of S^{t+1}, to lam_prev
    e = cudaMemcpyAsync(io, lam_next, sizeof(double) * n * NA, cudaMemcpyHostToDevice, ds.stream);
    if (e != cudaSuccess) return done(cuda_fail(c, e, "mpm_step_adjoint_1: copy lam_next"));
    c->aops->scatter_in(h, ds, NA, 0, order, io, a.lam[0]);
    {
        TimingScope ts(c, MPM_KERNEL_REVERSE);
        c->aops->step(h, ds, ad, st, GA, GV, GL, a.lam[0], a.lam[1], mub);
    }
    c->aops->gather(h, ds, NA, 0, order, a.lam[1], io);
    rc = check_launch(c, "mpm_step_adjoint_1");
    if (rc != MPM_OK) return done(rc);
    e = cudaMemcpyAsync(lam_prev, io, sizeof(double) * n * NA, cudaMemcpyDeviceToHost, ds.stream);
    if (e == cudaSuccess && wall >= 0)
        e = cudaMemcpyAsync(dL_dmu_out, a.d_mubar[wall],
                            sizeof(double) * ds.n_seg[wall][0] * ds.n_seg[wall][1], cudaMemcpyDeviceToHost, ds.stream);
    if (e != cudaSuccess) return done(cuda_fail(c, e, "mpm_step_adjoint_1: copy out"));
    return done(read_status(c));
}

int mpm_get_initial_adjoint(mpm_ctx *c, int field, double *out)
{
    if (!c || !out) return fail(c, MPM_EINVAL, "mpm_get_initial_adjoint: bad argument");
    AdjHost &a = c->adj;
    if (a.lam0 < 0) return fail(c, MPM_ESTATE, "mpm_get_initial_adjoint: no adjoint computed");
    const int d = c->grid.dim;
    int w = 0, off = 0;
    switch (field) {
    case MPM_FIELD_X: w = d; off = 0; break;
    case MPM_FIELD_V: w = d; off = d; break;
    case MPM_FIELD_C: w = d * d; off = 2 * d; break;
    case MPM_FIELD_RHO: w = 1; off = 2 * d + d * d; break;
    default: return fail(c, MPM_EINVAL, "mpm_get_initial_adjoint: field has no adjoint");
    }
    const int64_t n = c->hp.n;
    double *dev = nullptr;
    int rc = dalloc(c, &dev, (size_t)n * w, "initial adjoint");
    if (rc != MPM_OK) return rc;
    c->aops->gather(c->hp, c->ds, w, off, a.lam_id, a.lam[a.lam0], dev);
    cudaError_t e = cudaMemcpyAsync(out, dev, sizeof(double) * n * w, cudaMemcpyDeviceToHost, c->ds.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->ds.stream);
    dfree(dev);
    if (e != cudaSuccess) return fail(c, MPM_ECUDA, "mpm_get_initial_adjoint: copy failed");
    return MPM_OK;
}

int mpm_step_adjoint(mpm_ctx *c, int n_steps, int checkpoint_every, int wall, double *loss_out, double *dL_dmu_out)
{
    if (!c || n_steps < 1 || checkpoint_every < 1 || !loss_out || (wall >= 0 && !dL_dmu_out))
        return fail(c, MPM_EINVAL, "mpm_step_adjoint: bad argument");
    if (c->hp.n == 0) return fail(c, MPM_ESTATE, "mpm_step_adjoint: no particles loaded");
    if (c->grid.batch != 1) return fail(c, MPM_EINVAL, "mpm_step_adjoint: batch must be 1");
    if (c->grid.transfer != MPM_TRANSFER_APIC)
        return fail(c, MPM_EINVAL, "mpm_step_adjoint: the adjoint follows the APIC transfer");
    if (wall < -1 || wall >= 2 * c->grid.dim || (wall >= 0 && c->ds.mu_dev[wall] == nullptr))
        return fail(c, MPM_EINVAL, "mpm_step_adjoint: the wall has no friction field");
    AdjHost &a = c->adj;
    if (a.n_obs == 0 && a.n_mobs == 0) return fail(c, MPM_ESTATE, "mpm_step_adjoint: no observations set");
    if ((a.n_obs > 0 && a.steps.back() > n_steps) || (a.n_mobs > 0 && a.msteps.back() > n_steps))
        return fail(c, MPM_EINVAL, "mpm_step_adjoint: observation beyond the horizon");
    a.lam0 = -1;
    const HostParams &h = c->hp;
    DevState &ds = c->ds;
    const int d = h.dim;
    const int K = std::min(checkpoint_every, n_steps);
    const int NA = adj_ncomp_material(d, c->mat.kind == MPM_DRUCKER_PRAGER ? 1 : 0);
    const size_t rsz = h.precision == MPM_FP64 ? 8 : 4;
    const int64_t n = h.n;
    const size_t st_bytes = (size_t)NA * n * rsz;
    const int64_t n_ckpt = (n_steps + K - 1) / K;
    const size_t gbytes = (size_t)h.nodes_per_sim * 4 * rsz;
    const size_t fbytes = ((size_t)(h.node_tiles_per_sim + 1) * sizeof(int32_t) + 255) / 256 * 256;
    // cell-ordered v_bar scatter (3D single precision): coefficients and sort tables
    // for every sort generation a segment can hold
    const bool split = d == 3 && h.precision == MPM_FP32;
    const int gens_seg = std::min(K, K / std::max(1, c->grid.sort_every) + 2);
    const int64_t TNc = 512 + 1;
    const size_t gen_bytes = split ? (size_t)ds.max_tiles * (sizeof(int4) + TNc * 4) + (size_t)n * 4 + 4 : 0;
    // segments kept from the first pass: the last one always; more while the budget
    // set by mpm_set_adjoint_memory allows (those need no recomputation)
    const size_t seg_bytes = (size_t)K * (st_bytes + 2 * gbytes + fbytes + (size_t)n * 4) + gens_seg * gen_bytes;
    int64_t m_keep = 1 + (int64_t)(c->adj_budget > 0 ? c->adj_budget / (int64_t)seg_bytes : 0);
    if (m_keep > n_ckpt) m_keep = n_ckpt;
    // with one kept segment the reverse sweep of segment k runs on a second stream
    // while segment k - 1 is recomputed into the other of two banks of K slots
    const bool overlap = MPM_ADJ_OVERLAP && m_keep == 1 && n_ckpt >= 2;
    const int64_t banks = overlap ? 2 : m_keep;
    const int64_t KS = banks * K;                  // kept-state slots
    const int gens = split ? (int)(banks * gens_seg) : 0;
    {
        int rc = adj_buffers(c, n_ckpt, KS, gens);
        if (rc != MPM_OK) return rc;
    }
    MuBar mub{};
    for (int w = 0; w < kMaxWalls; ++w) {
        if (ds.mu_dev[w] == nullptr) continue;
        const int64_t cnt = (int64_t)ds.n_seg[w][0] * ds.n_seg[w][1];
        if (a.d_mubar[w] == nullptr) {
            int rc = dalloc(c, &a.d_mubar[w], cnt, "dL/dmu");
            if (rc != MPM_OK) return rc;
        }
        CK(cudaMemsetAsync(a.d_mubar[w], 0, sizeof(double) * cnt, ds.stream), "zero dL/dmu");
        mub.w[w] = a.d_mubar[w];
    }
    std::vector<int> obs_of_step(n_steps + 1, -1), mobs_of_step(n_steps + 1, -1);
    for (int o = 0; o < a.n_obs; ++o) obs_of_step[a.steps[o]] = o;
    for (int o = 0; o < a.n_mobs; ++o) mobs_of_step[a.msteps[o]] = o;
    const size_t msum_stride = (size_t)a.n_mon * (d + 1), mg_stride = (size_t)a.n_mon * d;
    if (a.n_mobs > 0)
        CK(cudaMemsetAsync(a.d_msums, 0, sizeof(double) * a.n_mobs * msum_stride, ds.stream), "zero monitor sums");
    auto ckpt_ptr = [&](int64_t k) { return (void *)((char *)a.ckpt + k * st_bytes); };
    auto seg_ptr = [&](int64_t j) { return (void *)((char *)a.seg + j * st_bytes); };
    auto gridA_ptr = [&](int64_t j) { return (void *)((char *)a.seg_grid + 2 * j * gbytes); };
    auto gridV_ptr = [&](int64_t j) { return (void *)((char *)a.seg_grid + (2 * j + 1) * gbytes); };
    auto gridL_ptr = [&](int64_t j) { return (int32_t *)((char *)a.seg_grid + 2 * KS * gbytes + j * fbytes); };
    // kept states live in slots: the last m_keep segments of the first pass in blocks
    // of K (segment n_ckpt - m_keep + b in block b), recomputed segments in block 0
    std::vector<int64_t> seg_gen(KS);
    std::vector<int> seg_ids(KS);               // which slot of seg_id holds the order of state j
    std::vector<int> seg_tab(KS, -1);           // which generation slot holds the sort tables of state j
    int next_gen = 0;
    auto seg_id_ptr = [&](int64_t j) { return a.seg_id + (int64_t)seg_ids[j] * n; };
    // state j of a segment: after the step's sort, P2G copies the state it reads and
    // the grid update saves its grid; the order's ids are copied once per sort
    auto keep_state = [&](int j, int jfirst, int gbase, int gend) -> int {
        if (c->need_sort || c->steps_since_sort >= c->grid.sort_every) {
            int rc = do_sort(c);
            if (rc != MPM_OK) return rc;
        }
        seg_gen[j] = c->sorts;
        if (j > jfirst && seg_gen[j] == seg_gen[j - 1]) {
            seg_ids[j] = seg_ids[j - 1];
            seg_tab[j] = seg_tab[j - 1];
        } else {
            seg_ids[j] = j;
            CK(cudaMemcpyAsync(a.seg_id + (int64_t)j * n, ds.id, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice,
                               ds.stream), "segment order");
            if (j == jfirst) next_gen = gbase;
            seg_tab[j] = -1;
            if (split && next_gen < gend) {            // the sort tables of this generation
                const int g = next_gen++;
                seg_tab[j] = g;
                CK(cudaMemcpyAsync(a.gen_tiles + (int64_t)g * ds.max_tiles, ds.tiles, sizeof(int4) * ds.max_tiles,
                                   cudaMemcpyDeviceToDevice, ds.stream), "generation tiles");
                CK(cudaMemcpyAsync(a.gen_ntiles + g, ds.counters + 1, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                   ds.stream), "generation tile count");
                CK(cudaMemcpyAsync(a.gen_posmap + (int64_t)g * n, ds.posmap, sizeof(int32_t) * n,
                                   cudaMemcpyDeviceToDevice, ds.stream), "generation position map");
                CK(cudaMemcpyAsync(a.gen_celloff + (int64_t)g * ds.max_tiles * TNc, ds.cell_off,
                                   sizeof(int32_t) * ds.max_tiles * TNc, cudaMemcpyDeviceToDevice, ds.stream),
                   "generation offsets");
            }
        }
        ds.save_S = seg_ptr(j);
        ds.save_A = gridA_ptr(j);
        ds.save_V = gridV_ptr(j);
        ds.save_L = gridL_ptr(j);
        return MPM_OK;
    };
    auto stop_keeping = [&]() {
        ds.save_S = ds.save_A = ds.save_V = nullptr;
        ds.save_L = nullptr;
    };
    CK(cudaMemsetAsync(a.grid.GVB, 0, gbytes, ds.stream), "zero grid adjoint");
    const size_t obs_stride = (size_t)a.n_track * d;
    // forward pass with checkpoints and observations; the last segment's states
    // and grids are kept on the way (its reverse needs no recompute)
    const int64_t first_kept = n_ckpt - m_keep;         // segments from here on are kept by the first pass
    const int64_t last_t0 = first_kept * K;
    c->aops->save(h, ds, ckpt_ptr(0));
    for (int t = 1; t <= n_steps; ++t) {
        if (t - 1 >= last_t0) {
            int rc = keep_state((int)(t - 1 - last_t0), 0, 0, overlap ? gens_seg : a.gen_cap);
            if (rc != MPM_OK) return rc;
        }
        int rc = step_many(c, 1);
        stop_keeping();
        if (rc != MPM_OK) return rc;
        if (obs_of_step[t] >= 0) c->aops->track(h, ds, a.d_track_of_id, a.d_xobs + obs_of_step[t] * obs_stride);
        if (mobs_of_step[t] >= 0) {
            const size_t rs = rsz * (size_t)kPB;
            c->aops->monitor_sum(h, ds, (char *)ds.S + rs * h.off_x, (char *)ds.S + rs * h.off_v, -h.ncomp, a.n_mon,
                                 a.d_mboxes, a.d_msums + mobs_of_step[t] * msum_stride);
        }
        if (t % K == 0 && t / K < first_kept) c->aops->save(h, ds, ckpt_ptr(t / K));   // recomputed later
    }
    CK(cudaMemcpyAsync(a.final_S, ds.S, ((size_t)h.ncomp * h.npad + 64) * rsz, cudaMemcpyDeviceToDevice, ds.stream),
       "save final state");
    CK(cudaMemcpyAsync(a.final_id, ds.id, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ds.stream), "save ids");
    CK(cudaMemcpyAsync(a.final_sim, ds.sim, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ds.stream), "save sims");
    std::vector<double> xobs((size_t)a.n_obs * obs_stride);
    CK(cudaMemcpyAsync(xobs.data(), a.d_xobs, sizeof(double) * xobs.size(), cudaMemcpyDeviceToHost, ds.stream),
       "copy observed positions");
    {
        int rc = read_status(c);
        if (rc != MPM_OK) return rc;
    }
    double loss = 0.0;
    for (size_t i = 0; i < xobs.size(); ++i) {
        const double e = xobs[i] - a.z[i];
        loss += e * e;
    }
    // monitor loss sum_obs sum_l |Q_l - z_l|^2 over non-empty monitors, and its seeds
    // g_l = 2 (Q_l - z_l) / |P_l|
    if (a.n_mobs > 0) {
        std::vector<double> ms(a.n_mobs * msum_stride), mg(a.n_mobs * mg_stride, 0.0);
        CK(cudaMemcpy(ms.data(), a.d_msums, sizeof(double) * ms.size(), cudaMemcpyDeviceToHost), "monitor sums");
        for (int o = 0; o < a.n_mobs; ++o)
            for (int l = 0; l < a.n_mon; ++l) {
                const double *sm = &ms[o * msum_stride + (size_t)l * (d + 1)];
                const double cnt = sm[d];
                if (!(cnt > 0.0)) continue;
                for (int b = 0; b < d; ++b) {
                    const double e = sm[b] / cnt - a.mz[o * mg_stride + (size_t)l * d + b];
                    loss += e * e;
                    mg[o * mg_stride + (size_t)l * d + b] = 2.0 * e / cnt;
                }
            }
        CK(cudaMemcpy(a.d_mg, mg.data(), sizeof(double) * mg.size(), cudaMemcpyHostToDevice), "monitor seeds");
    }
    // Reverse sweep, one segment at a time (recomputed from its checkpoint).  States
    // are saved in the particle order the context holds at the time (a contiguous
    // copy); the adjoint state follows the order of the state it belongs to and is
    // re-ordered only where a sort changed the order between two states.
    int cur = 0;
    int64_t lam_gen = c->sorts;                // the order of the final state
    CK(cudaMemcpyAsync(a.lam_id, ds.id, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ds.stream), "adjoint order");
    c->aops->zero(h, ds, a.lam[cur], (int64_t)NA * n);
    if (obs_of_step[n_steps] >= 0) {
        const int o = obs_of_step[n_steps];
        c->aops->seed_slots(h, ds, a.lam_id, a.d_track_of_id, a.d_xobs + o * obs_stride, a.d_z + o * obs_stride,
                            a.lam[cur]);
    }
    if (mobs_of_step[n_steps] >= 0) {               // the final state's positions, in the order of lam
        const size_t rs = rsz * (size_t)kPB;
        c->aops->monitor_seed(h, ds, (char *)ds.S + rs * h.off_x, -h.ncomp, a.n_mon, a.d_mboxes,
                              a.d_mg + mobs_of_step[n_steps] * mg_stride, a.lam[cur]);
    }
    // With overlap the reverse steps run on a second stream: while segment k is
    // reversed there from one bank, segment k - 1 is recomputed on the context's
    // stream into the other bank, once the reverse of segment k + 1 has released it.
    cudaStream_t rstream = ds.stream;
    if (overlap) {
        if (a.rstream == nullptr) {
            // (giving it the highest stream priority measured no different: 445.0 against
            // 445.2 ms on the 1.36M-particle problem)
            CK(cudaStreamCreateWithFlags(&a.rstream, cudaStreamNonBlocking), "reverse stream");
            for (int b = 0; b < 2; ++b) {
                CK(cudaEventCreateWithFlags(&a.ev_filled[b], cudaEventDisableTiming), "bank event");
                CK(cudaEventCreateWithFlags(&a.ev_read[b], cudaEventDisableTiming), "bank event");
            }
        }
        rstream = a.rstream;
    }
    DevState dr = ds;                                 // the reverse steps' launch state
    dr.stream = rstream;
    auto bank_of = [&](int64_t k) { return overlap ? (int)((n_ckpt - 1 - k) % 2) : 0; };
    // recompute segment k from its checkpoint into its bank (on the context's stream)
    auto recompute = [&](int64_t k) -> int {
        const int t0 = (int)(k * K), t1 = (int)std::min<int64_t>((k + 1) * K, n_steps);
        const int bk = bank_of(k), s0 = bk * K;
        const int g0 = overlap ? bk * gens_seg : 0, g1 = overlap ? g0 + gens_seg : a.gen_cap;
        c->aops->restore(h, ds, ckpt_ptr(k));
        c->need_sort = true;
        for (int j = 0; j < t1 - t0; ++j) {
            int rc = keep_state(s0 + j, s0, g0, g1);
            if (rc == MPM_OK) rc = step_many(c, 1);
            stop_keeping();
            if (rc != MPM_OK) return rc;
        }
        return MPM_OK;
    };
    // on an error the reverse stream is drained before returning
    auto join = [&](int rc) {
        if (overlap) cudaStreamSynchronize(rstream);
        return rc;
    };
    if (overlap) CK(cudaEventRecord(a.ev_filled[0], ds.stream), "bank event");   // the last segment and the seeds
    for (int64_t k = n_ckpt - 1; k >= 0; --k) {
        const int t0 = (int)(k * K), t1 = (int)std::min<int64_t>((k + 1) * K, n_steps);
        int base;                                      // slot of the segment's first state
        if (overlap) {
            if (k >= 1) {
                const int bn = bank_of(k - 1);
                if (k + 1 <= n_ckpt - 1) CK(cudaStreamWaitEvent(ds.stream, a.ev_read[bn], 0), "bank wait");
                int rc = recompute(k - 1);
                if (rc != MPM_OK) return join(rc);
                CK(cudaEventRecord(a.ev_filled[bn], ds.stream), "bank event");
            }
            CK(cudaStreamWaitEvent(rstream, a.ev_filled[bank_of(k)], 0), "bank wait");
            base = bank_of(k) * K;
        } else {
            base = k >= first_kept ? (int)((k - first_kept) * K) : 0;
            if (k < first_kept) {
                int rc = recompute(k);
                if (rc != MPM_OK) return rc;
            }
        }
        for (int t = t1 - 1; t >= t0; --t) {
            const int j = base + t - t0;               // the kept state's slot
            if (seg_gen[j] != lam_gen) {             // a sort between the two states: re-order
                c->aops->reorder(h, dr, NA, a.lam_id, a.lam_pos, seg_id_ptr(j), a.lam[cur], a.lam[cur ^ 1]);
                cur ^= 1;
                CK(cudaMemcpyAsync(a.lam_id, seg_id_ptr(j), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice,
                                   rstream), "adjoint order");
                lam_gen = seg_gen[j];
            }
            AdjDev ad = a.grid;
            if (seg_tab[j] >= 0) {
                const int g = seg_tab[j];
                ad.coef = a.coef;
                ad.cursor = ds.counters + 5;
                ad.tiles = a.gen_tiles + (int64_t)g * ds.max_tiles;
                ad.n_tiles = a.gen_ntiles + g;
                ad.posmap = a.gen_posmap + (int64_t)g * n;
                ad.cell_off = a.gen_celloff + (int64_t)g * ds.max_tiles * TNc;
            }
            {
                TimingScope ts(c, MPM_KERNEL_REVERSE, rstream);
                c->aops->step(h, dr, ad, seg_ptr(j), gridA_ptr(j), gridV_ptr(j), gridL_ptr(j), a.lam[cur],
                              a.lam[cur ^ 1], mub);
            }
            cur ^= 1;
            if (t >= 1 && obs_of_step[t] >= 0) {
                const int o = obs_of_step[t];
                c->aops->seed_slots(h, dr, a.lam_id, a.d_track_of_id, a.d_xobs + o * obs_stride,
                                    a.d_z + o * obs_stride, a.lam[cur]);
            }
            if (t >= 1 && mobs_of_step[t] >= 0)     // S^t is the state kept for step j, in the order of lam
                c->aops->monitor_seed(h, dr, seg_ptr(j), n, a.n_mon, a.d_mboxes,
                                      a.d_mg + mobs_of_step[t] * mg_stride, a.lam[cur]);
        }
        if (overlap) CK(cudaEventRecord(a.ev_read[bank_of(k)], rstream), "bank event");
        int rc = check_launch(c, "mpm_step_adjoint");
        if (rc != MPM_OK) return join(rc);
    }
    if (overlap) CK(cudaStreamWaitEvent(ds.stream, a.ev_read[bank_of(0)], 0), "join the reverse stream");
    // leave the context at the end-of-horizon state
    CK(cudaMemcpyAsync(ds.S, a.final_S, ((size_t)h.ncomp * h.npad + 64) * rsz, cudaMemcpyDeviceToDevice, ds.stream),
       "restore final state");
    CK(cudaMemcpyAsync(ds.id, a.final_id, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ds.stream), "restore ids");
    CK(cudaMemcpyAsync(ds.sim, a.final_sim, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ds.stream),
       "restore sims");
    c->need_sort = true;
    a.lam0 = cur;
    if (wall >= 0) {
        const int64_t cnt = (int64_t)ds.n_seg[wall][0] * ds.n_seg[wall][1];
        CK(cudaMemcpyAsync(dL_dmu_out, a.d_mubar[wall], sizeof(double) * cnt, cudaMemcpyDeviceToHost, ds.stream),
           "copy dL/dmu");
    }
    int rc = read_status(c);
    if (rc != MPM_OK) return rc;
    *loss_out = loss;
    return MPM_OK;
}

int mpm_save_state(mpm_ctx *c, int slot)
{
    if (!c || slot < 0 || slot >= kMaxSlots) return fail(c, MPM_EINVAL, "mpm_save_state: bad slot");
    if (c->hp.n == 0) return fail(c, MPM_ESTATE, "mpm_save_state: no particles loaded");
    const HostParams &h = c->hp;
    StateSlot &sl = c->slots[slot];
    const size_t bytes = ((size_t)h.ncomp * h.npad + 64) * (h.precision == MPM_FP64 ? 8 : 4);
    if (sl.n != h.n) {
        dfree(sl.S); dfree(sl.id); dfree(sl.sim);
        int rc = dalloc(c, (unsigned char **)&sl.S, bytes, "state slot");
        if (rc == MPM_OK) rc = dalloc(c, &sl.id, h.n, "state slot ids");
        if (rc == MPM_OK) rc = dalloc(c, &sl.sim, h.n, "state slot sims");
        if (rc != MPM_OK) {
            sl.n = 0;
            return rc;
        }
        sl.n = h.n;
    }
    DevState &ds = c->ds;
    CK(cudaMemcpyAsync(sl.S, ds.S, bytes, cudaMemcpyDeviceToDevice, ds.stream), "save state");
    CK(cudaMemcpyAsync(sl.id, ds.id, sizeof(int32_t) * h.n, cudaMemcpyDeviceToDevice, ds.stream), "save ids");
    CK(cudaMemcpyAsync(sl.sim, ds.sim, sizeof(int32_t) * h.n, cudaMemcpyDeviceToDevice, ds.stream), "save sims");
    return MPM_OK;
}

int mpm_restore_state(mpm_ctx *c, int slot)
{
    if (!c || slot < 0 || slot >= kMaxSlots) return fail(c, MPM_EINVAL, "mpm_restore_state: bad slot");
    const HostParams &h = c->hp;
    StateSlot &sl = c->slots[slot];
    if (h.n == 0 || sl.n != h.n) return fail(c, MPM_ESTATE, "mpm_restore_state: slot is empty");
    const size_t bytes = ((size_t)h.ncomp * h.npad + 64) * (h.precision == MPM_FP64 ? 8 : 4);
    DevState &ds = c->ds;
    CK(cudaMemcpyAsync(ds.S, sl.S, bytes, cudaMemcpyDeviceToDevice, ds.stream), "restore state");
    CK(cudaMemcpyAsync(ds.id, sl.id, sizeof(int32_t) * h.n, cudaMemcpyDeviceToDevice, ds.stream), "restore ids");
    CK(cudaMemcpyAsync(ds.sim, sl.sim, sizeof(int32_t) * h.n, cudaMemcpyDeviceToDevice, ds.stream), "restore sims");
    c->need_sort = true;
    return MPM_OK;
}

namespace {
// FNV-1a 64-bit hash (Fowler-Noll-Vo) of a byte range.
uint64_t fnv1a(const unsigned char *p, size_t n, uint64_t h = 1469598103934665603ull)
{
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}
struct BlobHeader {
    uint64_t magic, n, ncomp, npad, precision, dim, payload, checksum;
};
constexpr uint64_t kBlobMagic = 0x4d504d5354415445ull;   // "MPMSTATE"
// One component of the blocked particle state to or from n consecutive host
// values: a strided copy over the whole blocks of kPB particles, then the tail.
cudaError_t copy_component(const HostParams &h, int comp, char *S, char *host, bool to_device, cudaStream_t st)
{
    const size_t rs = h.precision == MPM_FP64 ? 8 : 4;
    const size_t row = kPB * rs, pitch = (size_t)h.ncomp * kPB * rs;
    const int64_t nfull = h.n / kPB, rem = h.n % kPB;
    char *dev = S + (size_t)comp * kPB * rs;
    cudaError_t e = cudaSuccess;
    if (nfull > 0)
        e = to_device ? cudaMemcpy2DAsync(dev, pitch, host, row, row, (size_t)nfull, cudaMemcpyHostToDevice, st)
                      : cudaMemcpy2DAsync(host, row, dev, pitch, row, (size_t)nfull, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && rem > 0) {
        char *dt = dev + (size_t)nfull * pitch, *ht = host + (size_t)nfull * row;
        e = to_device ? cudaMemcpyAsync(dt, ht, (size_t)rem * rs, cudaMemcpyHostToDevice, st)
                      : cudaMemcpyAsync(ht, dt, (size_t)rem * rs, cudaMemcpyDeviceToHost, st);
    }
    return e;
}

}  // namespace

int64_t mpm_state_blob_size(const mpm_ctx *c)
{
    if (!c || c->hp.n == 0) return MPM_ESTATE;
    const HostParams &h = c->hp;
    const int64_t rs = h.precision == MPM_FP64 ? 8 : 4;
    return (int64_t)sizeof(BlobHeader) + (int64_t)h.ncomp * h.n * rs + 2 * h.n * (int64_t)sizeof(int32_t);
}

int mpm_export_state(mpm_ctx *c, void *blob, int64_t size)
{
    if (!c || !blob) return fail(c, MPM_EINVAL, "mpm_export_state: bad argument");
    const int64_t need = mpm_state_blob_size(c);
    if (need < 0) return fail(c, MPM_ESTATE, "mpm_export_state: no particles loaded");
    if (size < need) return fail(c, MPM_EINVAL, "mpm_export_state: buffer too small");
    const HostParams &h = c->hp;
    DevState &ds = c->ds;
    const int64_t rs = h.precision == MPM_FP64 ? 8 : 4;
    BlobHeader hd{kBlobMagic, (uint64_t)h.n, (uint64_t)h.ncomp, (uint64_t)h.npad, (uint64_t)h.precision,
                  (uint64_t)h.dim, (uint64_t)(need - (int64_t)sizeof(BlobHeader)), 0};
    unsigned char *out = (unsigned char *)blob + sizeof(BlobHeader);
    for (int comp = 0; comp < h.ncomp; ++comp)
        CK(copy_component(h, comp, (char *)ds.S, (char *)out + (size_t)comp * h.n * rs, false, ds.stream),
           "export state");
    unsigned char *ids = out + (size_t)h.ncomp * h.n * rs;
    CK(cudaMemcpyAsync(ids, ds.id, sizeof(int32_t) * h.n, cudaMemcpyDeviceToHost, ds.stream), "export ids");
    CK(cudaMemcpyAsync(ids + sizeof(int32_t) * h.n, ds.sim, sizeof(int32_t) * h.n, cudaMemcpyDeviceToHost, ds.stream),
       "export sims");
    CK(cudaStreamSynchronize(ds.stream), "export state");
    hd.checksum = fnv1a(out, hd.payload);
    std::memcpy(blob, &hd, sizeof hd);
    return MPM_OK;
}

int mpm_import_state(mpm_ctx *c, const void *blob, int64_t size)
{
    if (!c || !blob || size < (int64_t)sizeof(BlobHeader)) return fail(c, MPM_EINVAL, "mpm_import_state: bad argument");
    BlobHeader hd;
    std::memcpy(&hd, blob, sizeof hd);
    const HostParams &h = c->hp;
    if (hd.magic != kBlobMagic) return fail(c, MPM_ECORRUPT, "mpm_import_state: not a state blob");
    if (h.n == 0 || hd.n != (uint64_t)h.n || hd.ncomp != (uint64_t)h.ncomp || hd.precision != (uint64_t)h.precision ||
        hd.dim != (uint64_t)h.dim)
        return fail(c, MPM_EINVAL, "mpm_import_state: blob does not match the loaded particles");
    const int64_t rs = h.precision == MPM_FP64 ? 8 : 4;
    const uint64_t expect = (uint64_t)h.ncomp * h.n * rs + 2 * sizeof(int32_t) * (uint64_t)h.n;
    if (hd.payload != expect) return fail(c, MPM_ECORRUPT, "mpm_import_state: payload size does not match");
    if ((int64_t)(sizeof(BlobHeader) + hd.payload) > size) return fail(c, MPM_ECORRUPT, "mpm_import_state: truncated");
    const unsigned char *in = (const unsigned char *)blob + sizeof(BlobHeader);
    if (fnv1a(in, hd.payload) != hd.checksum) return fail(c, MPM_ECORRUPT, "mpm_import_state: checksum mismatch");
    // the ids index the load-order readback and the simulation ids the per-simulation
    // grids: a blob whose ids are not a permutation of 0..n-1, or whose simulation ids
    // leave the batch, is refused before anything reaches the device
    std::vector<int32_t> ids(h.n), sims(h.n);
    std::memcpy(ids.data(), in + (size_t)h.ncomp * h.n * rs, sizeof(int32_t) * h.n);
    std::memcpy(sims.data(), in + (size_t)h.ncomp * h.n * rs + sizeof(int32_t) * h.n, sizeof(int32_t) * h.n);
    {
        std::vector<unsigned char> seen(h.n, 0);
        for (int64_t p = 0; p < h.n; ++p) {
            if (ids[p] < 0 || ids[p] >= h.n || seen[ids[p]])
                return fail(c, MPM_ECORRUPT, "mpm_import_state: particle ids are not a permutation");
            seen[ids[p]] = 1;
            if (sims[p] < 0 || sims[p] >= c->grid.batch)
                return fail(c, MPM_ECORRUPT, "mpm_import_state: simulation id out of range");
        }
    }
    DevState &ds = c->ds;
    for (int comp = 0; comp < h.ncomp; ++comp)
        CK(copy_component(h, comp, (char *)ds.S, (char *)in + (size_t)comp * h.n * rs, true, ds.stream),
           "import state");
    CK(cudaMemcpyAsync(ds.id, ids.data(), sizeof(int32_t) * h.n, cudaMemcpyHostToDevice, ds.stream), "import ids");
    CK(cudaMemcpyAsync(ds.sim, sims.data(), sizeof(int32_t) * h.n, cudaMemcpyHostToDevice, ds.stream), "import sims");
    CK(cudaStreamSynchronize(ds.stream), "import state");
    c->need_sort = true;
    return MPM_OK;
}

}  // extern "C"
