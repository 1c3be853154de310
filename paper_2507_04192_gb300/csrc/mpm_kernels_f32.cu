// Instantiation of the MPM kernels for float arithmetic.
#include "mpm_kernels.cuh"

namespace mpm {

const Ops ops_f32 = {
    Dispatch<float>::init_state, Dispatch<float>::keys,      Dispatch<float>::permute,
    Dispatch<float>::p2g,        Dispatch<float>::grid,      Dispatch<float>::g2p,
    Dispatch<float>::get_field,  Dispatch<float>::set_field,
};

}  // namespace mpm
