// Instantiation of the MPM kernels for double arithmetic.
#include "mpm_kernels.cuh"

namespace mpm {

const Ops ops_f64 = {
    Dispatch<double>::init_state, Dispatch<double>::keys,      Dispatch<double>::permute,
    Dispatch<double>::p2g,        Dispatch<double>::grid,      Dispatch<double>::g2p,
    Dispatch<double>::get_field,  Dispatch<double>::set_field,
};

}  // namespace mpm
