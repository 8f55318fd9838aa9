// Allocation-free time stepping: plb_step_pairs_static (include/plb.h).
//
// Some callers cannot allocate device memory at all: a plugin that runs inside another
// framework's memory arena and is handed only the buffers it works on, or a real-time loop
// in which a cudaMalloc (which may synchronise the device) is forbidden.  For them this
// entry point advances a caller-owned population array using the same psi-pass and
// force/collide/stream kernels as plb_step, with the only scratch they need (the padded
// psi field and the error flags) held in a fixed file-scope device array.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "plb.h"
#include "plb_host.h"
#include "plb_launch.h"

namespace {
constexpr size_t kScratchBytes = size_t(8) << 20;   // 8 MiB per device, held until exit
constexpr size_t kFlagBytes = 256;                   // last 256 bytes: device error flags
constexpr int kMaxDevices = 64;
}  // namespace

// Device scratch of plb_step_pairs_static.  In host code this name is only a stand-in for
// the symbol; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_plb_static_scratch[kScratchBytes];

namespace {
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices];

// Device address of the scratch array on the current device, looked up once per device.
int scratch_address(void **addr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return plb::set_error(PLB_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return plb::set_error(PLB_EUNSUPPORTED, "device %d: at most %d devices are supported", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_plb_static_scratch);
        if (e != cudaSuccess || !p)
            return plb::set_error(PLB_ECUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    return PLB_OK;
}
}  // namespace

extern "C" int plb_step_pairs_static(int lattice, const int dims[3], const plb_eos_params *eos, double tau, double G,
                                     double eps, const plb_opts *opts, void *dev_pops, int npairs, long long t0,
                                     void *cuda_stream) {
    plb_opts o;
    plb::Layout lay;
    int st = plb::check_create_args(lattice, dims, eos, tau, G, eps, opts, o, lay);
    if (st != PLB_OK) return st;
    if (o.streaming != PLB_STREAM_AA) return plb::set_error(PLB_EUNSUPPORTED, "this entry point steps in place (AA)");
    if (o.wall_y && o.wall_rho > 0.0)
        return plb::set_error(PLB_EUNSUPPORTED, "this entry point has neutral walls only (wall_rho <= 0)");
    if (!dev_pops) return plb::set_error(PLB_EINVAL, "dev_pops is NULL");
    if (reinterpret_cast<uintptr_t>(dev_pops) % 256 != 0)
        return plb::set_error(PLB_EINVAL, "dev_pops must be 256-byte aligned");
    if (npairs < 0) return plb::set_error(PLB_EINVAL, "npairs must be >= 0");
    if (t0 < 0) return plb::set_error(PLB_EINVAL, "t0 must be >= 0");
    const size_t psi_bytes = (size_t)lay.psi_elems * lay.s_psi;
    if (psi_bytes > kScratchBytes - kFlagBytes)
        return plb::set_error(PLB_ENOMEM,
                              "lattice too large for the static scratch: its padded psi field needs %zu bytes, the "
                              "limit is %zu bytes (about %zu cells in FP32/FP16S storage, %zu in FP64)",
                              psi_bytes, kScratchBytes - kFlagBytes, (kScratchBytes - kFlagBytes) / 4,
                              (kScratchBytes - kFlagBytes) / 8);
    void *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != PLB_OK) return st;

    double rv = 0, rl = 0, p0 = 0;
    if (plb::solve_coexistence(*eos, rv, rl, p0) != PLB_OK) rv = rl = 0;
    plb::KParams k;
    st = plb::fill_kparams(dims, *eos, tau, G, eps, o, lay, rv, rl, k);
    if (st != PLB_OK) return st;
    k.pstride = lay.n;   // the caller's planes are contiguous: f[i * N + s]
    k.flags = reinterpret_cast<unsigned *>(static_cast<char *>(scratch) + kScratchBytes - kFlagBytes);
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const plb::Launchers *L = plb::launchers_for_precision(lattice, o.precision);
    const int coll = o.collision == PLB_MRT ? 1 : 0;

    // An error left pending by earlier work on this thread would otherwise be reported below
    // as a failure of these launches.
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess)
        return plb::set_error(PLB_ECUDA, "a CUDA error from earlier work is pending on this thread: %s",
                              cudaGetErrorString(e));
    // The scratch keeps the previous call's contents: the flags must start at zero.
    e = cudaMemsetAsync(k.flags, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return plb::set_error(PLB_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    for (int n = 0; n < npairs; ++n) {
        for (int odd = 0; odd < 2; ++odd) {
            // the step counter seeds stochastic rounding exactly as plb_step does
            k.salt = (unsigned)(t0 + 2LL * n + odd);
            L->psi(k, dev_pops, scratch, odd, stream);
            L->collide[coll](k, dev_pops, scratch, odd, stream);
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return plb::set_error(PLB_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    unsigned flags = 0;
    e = cudaMemcpyAsync(&flags, k.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return plb::set_error(PLB_ECUDA, "reading the device flags: %s", cudaGetErrorString(e));
    if (flags & plb::FLAG_NONFINITE) return plb::set_error(PLB_ENONFINITE, "a density became non-positive or non-finite");
    if (flags & plb::FLAG_PSI_DOMAIN) return plb::set_error(PLB_EPSI_DOMAIN, "2 (p_EOS - rho/3) / G < 0 on some cell");
    return PLB_OK;
}
