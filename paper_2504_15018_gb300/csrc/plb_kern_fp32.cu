// Kernel instantiations for float population storage.
#include "plb_kernels.cuh"

namespace plb {

const Launchers *launchers_fp32(int lattice) {
    static const Launchers d2q9 = Launch<D2Q9, float>::table();
    static const Launchers d3q19 = Launch<D3Q19, float>::table();
    return lattice == 0 ? &d2q9 : &d3q19;
}

}  // namespace plb
