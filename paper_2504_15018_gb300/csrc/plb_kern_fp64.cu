// Kernel instantiations for double population storage.
#include "plb_kernels.cuh"

namespace plb {

const Launchers *launchers_fp64(int lattice) {
    static const Launchers d2q9 = Launch<D2Q9, double>::table();
    static const Launchers d3q19 = Launch<D3Q19, double>::table();
    return lattice == 0 ? &d2q9 : &d3q19;
}

}  // namespace plb
