// Instantiation of the MPM kernels for float arithmetic.
#include "mpm_adjoint.cuh"

namespace mpm {

const Ops ops_f32 = {
    Dispatch<float>::init_state, Dispatch<float>::keys,      Dispatch<float>::permute,
    Dispatch<float>::p2g,        Dispatch<float>::grid,      Dispatch<float>::g2p,
    Dispatch<float>::get_field,  Dispatch<float>::set_field, Dispatch<float>::diag_particles,
};

const AdjOps adj_ops_f32 = {
    AdjDispatch<float>::save, AdjDispatch<float>::restore, AdjDispatch<float>::track,
    AdjDispatch<float>::seed, AdjDispatch<float>::step,    AdjDispatch<float>::zero,
    AdjDispatch<float>::reorder, AdjDispatch<float>::seed_slots, AdjDispatch<float>::monitor_sum,
    AdjDispatch<float>::monitor_seed, AdjDispatch<float>::gather, AdjDispatch<float>::scatter_in,
};

}  // namespace mpm
