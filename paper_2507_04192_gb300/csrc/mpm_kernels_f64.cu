// Instantiation of the MPM kernels for double arithmetic.
#include "mpm_adjoint.cuh"

namespace mpm {

const Ops ops_f64 = {
    Dispatch<double>::init_state, Dispatch<double>::keys,      Dispatch<double>::permute,
    Dispatch<double>::p2g,        Dispatch<double>::grid,      Dispatch<double>::g2p,
    Dispatch<double>::get_field,  Dispatch<double>::set_field, Dispatch<double>::diag_particles,
};

const AdjOps adj_ops_f64 = {
    AdjDispatch<double>::save, AdjDispatch<double>::restore, AdjDispatch<double>::track,
    AdjDispatch<double>::seed, AdjDispatch<double>::step,    AdjDispatch<double>::zero,
    AdjDispatch<double>::reorder, AdjDispatch<double>::seed_slots, AdjDispatch<double>::monitor_sum,
    AdjDispatch<double>::monitor_seed, AdjDispatch<double>::gather, AdjDispatch<double>::scatter_in,
};

}  // namespace mpm
