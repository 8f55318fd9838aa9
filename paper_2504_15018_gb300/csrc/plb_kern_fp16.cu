// Kernel instantiations for __half population storage.
#include "plb_kernels.cuh"

namespace plb {

const Launchers *launchers_fp16(int lattice) {
    static const Launchers d2q9 = Launch<D2Q9, __half>::table();
    static const Launchers d3q19 = Launch<D3Q19, __half>::table();
    return lattice == 0 ? &d2q9 : &d3q19;
}

}  // namespace plb
