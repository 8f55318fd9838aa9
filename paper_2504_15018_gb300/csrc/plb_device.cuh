// Device-side building blocks of the P-LBM step (arXiv 2504.15018, Sec. II).
//
// Storage: populations in one copy, structure of arrays A[i * pstride + s]
// (s = x + nx (y + ny z)), updated in place with the AA pattern:
//   even parity  (natural layout)  read f_i(x) = A[i][x],             write f*_i -> A[opp i][x]
//   odd parity   (swapped layout)  read f_i(x) = A[opp i][x - c_i],   write f*_i -> A[i][x + c_i]
// Halfway bounce-back at the y walls: an odd-parity read from a wall cell becomes
// A[i][x] (the bounced f*_opp(i) stored there on the even step), and an odd-parity write
// into a wall becomes A[opp i][x].  Each thread reads and writes the same Q locations,
// so the update needs no second array and no inter-thread ordering.
//
// psi lives in a padded array with one ghost layer per side (x padded to a 16-byte
// multiple): the psi pass writes the periodic images, or the mirrored wall values, into
// the ghosts, so the force stencil never wraps.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "plb_f2.cuh"
#include "plb_launch.h"

namespace plb {

// ------------------------------------------------------------------ lattices
// Opposite directions are adjacent: opp(i) = i + 1 for odd i, i - 1 for even i > 0.
struct D2Q9 {
    static constexpr int Q = 9, D = 2;
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
};

struct D3Q19 {
    static constexpr int Q = 19, D = 3;
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i) {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
};

// Weights used by the collision in a reduced-precision type R.  The FP32 roundings of 1/36,
// 1/18 (or 1/9) and 1/3 (or 4/9) sum to 1 + 2^-27 (D2Q9) or 1 + 2^-26 (D3Q19); a relaxation
// toward an equilibrium whose weights do not sum to one changes the cell's mass by that
// fraction, the same sign every step, so FP32 lattices gained about 1e-8 of their mass per step.
// Here w(|c|^2 = 2) is 1/36 rounded to an FP32 value with an even significand, the |c|^2 = 1
// weight is a power-of-two multiple of it, and the rest weight is one minus the others; all
// three are exact FP32 values (the even significand makes the difference representable) and
// they sum to exactly one.  FP64 keeps the plain weights.
template <class L, class R>
__host__ __device__ constexpr double wcol(int i) {
    if (sizeof(R) == sizeof(double)) return L::w(i);
    constexpr double w2 = 0x1.c71c70p-6;                       // 1/36 (1 - 2.1e-7)
    constexpr double r1 = L::Q == 9 ? 4.0 : 2.0;               // w(|c|=1) / w(|c|^2=2)
    constexpr int n1 = L::Q == 9 ? 4 : 6, n2 = L::Q == 9 ? 4 : 12;
    const int c2 = L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i);
    return c2 == 0 ? 1.0 - n1 * r1 * w2 - n2 * w2 : (c2 == 1 ? r1 * w2 : w2);
}

__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// ------------------------------------------------------------ MRT moment bases
// Rows of the orthogonal bases as polynomials of c (Lallemand & Luo 2000 for D2Q9,
// d'Humieres et al. 2002 for D3Q19).  Only the non-hydrodynamic rows are needed
// here; kind tells which rate relaxes the row: 1 = s_e, 2 = s_eps, 3 = s_q, 4 = s_pi, 5 = s_m.
template <class L> struct Ghosts;

template <> struct Ghosts<D2Q9> {
    static constexpr int K = 4;
    __host__ __device__ static constexpr int kind(int k) {
        constexpr int t[4] = {1, 2, 3, 3};
        return t[k];
    }
    __host__ __device__ static constexpr double row(int k, int i) {
        double x = D2Q9::cx(i), y = D2Q9::cy(i), c2 = x * x + y * y;
        return k == 0 ? -4.0 + 3.0 * c2
             : k == 1 ? 4.0 - 10.5 * c2 + 4.5 * c2 * c2
             : k == 2 ? (-5.0 + 3.0 * c2) * x
                      : (-5.0 + 3.0 * c2) * y;
    }
};

template <> struct Ghosts<D3Q19> {
    static constexpr int K = 10;
    __host__ __device__ static constexpr int kind(int k) {
        constexpr int t[10] = {1, 2, 3, 3, 3, 4, 4, 5, 5, 5};
        return t[k];
    }
    __host__ __device__ static constexpr double row(int k, int i) {
        double x = D3Q19::cx(i), y = D3Q19::cy(i), z = D3Q19::cz(i), c2 = x * x + y * y + z * z;
        return k == 0 ? 19.0 * c2 - 30.0
             : k == 1 ? (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0
             : k == 2 ? (5.0 * c2 - 9.0) * x
             : k == 3 ? (5.0 * c2 - 9.0) * y
             : k == 4 ? (5.0 * c2 - 9.0) * z
             : k == 5 ? (3.0 * c2 - 5.0) * (3.0 * x * x - c2)
             : k == 6 ? (3.0 * c2 - 5.0) * (y * y - z * z)
             : k == 7 ? (y * y - z * z) * x
             : k == 8 ? (z * z - x * x) * y
                      : (x * x - y * y) * z;
    }
};

template <class L> __host__ __device__ constexpr double row_norm2(int k) {
    double n = 0.0;
    for (int i = 0; i < L::Q; ++i) n += Ghosts<L>::row(k, i) * Ghosts<L>::row(k, i);
    return n;
}

// ----------------------------------------------------------- storage traits
// Arithmetic in double for FP64 storage, float otherwise.  ld / st move one stored value
// to / from arithmetic precision without any shift; with SHIFT (FP16 storage) the stored
// value is the deviation f_i - w_i rho_ref, and the kernels account for the shift.
// Load policies.  LdStream: populations streamed with evict-first hints, psi through the
// read-only path; right for kernels in which nothing read is written by another block.
// LdCoherent: every load through L2 only, for the persistent batch kernel, whose blocks read
// across grid barriers what other SMs wrote in the same launch (L1 is not coherent).
struct LdStream {
    template <class U> __device__ __forceinline__ static U ld(const U *a) { return __ldcs(a); }
    template <class U> __device__ __forceinline__ static U ro(const U *a) { return __ldg(a); }
};
struct LdCoherent {
    template <class U> __device__ __forceinline__ static U ld(const U *a) { return __ldcg(a); }
    template <class U> __device__ __forceinline__ static U ro(const U *a) { return __ldcg(a); }
};
// LdKeep: loads of data the same kernel reads again shortly (the single-pass kernel reads a
// plane's populations for psi, then once more a plane later for the collision): L2
// evict-last priority through a createpolicy cache hint.
struct LdKeep {
    __device__ __forceinline__ static unsigned ld(const unsigned *a) {
        unsigned v;
        asm("{\n\t.reg .b64 pol;\n\tcreatepolicy.fractional.L2::evict_last.b64 pol, 1.0;\n\t"
            "ld.global.L2::cache_hint.b32 %0, [%1], pol;\n\t}"
            : "=r"(v) : "l"(a));
        return v;
    }
    __device__ __forceinline__ static float2 ld(const float2 *a) {
        float2 v;
        asm("{\n\t.reg .b64 pol;\n\tcreatepolicy.fractional.L2::evict_last.b64 pol, 1.0;\n\t"
            "ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], pol;\n\t}"
            : "=f"(v.x), "=f"(v.y) : "l"(a));
        return v;
    }
    template <class U> __device__ __forceinline__ static U ro(const U *a) { return __ldg(a); }
};
// LdBatch: the persistent batch kernel after a grid barrier.  The barrier is a release /
// acquire pattern at GPU scope (atomic arrival and __threadfence on both sides, then a block
// barrier), so ordinary L1-cached loads issued after it observe the other blocks' writes.
// Populations are read once and bypass L1; the psi stencil, read by several threads, is cached.
struct LdBatch {
    template <class U> __device__ __forceinline__ static U ld(const U *a) { return __ldcg(a); }
    template <class U> __device__ __forceinline__ static U ro(const U *a) { return __ldca(a); }
};

template <class S> struct Store;
template <> struct Store<double> {
    using T = double;
    using PsiT = double;
    static constexpr bool SHIFT = false;
    template <class Pol = LdStream> __device__ static T ld(const double *a) { return Pol::ld(a); }
    __device__ static void st(double *a, T v) { __stcs(a, v); }
};
template <> struct Store<float> {
    using T = float;
    using PsiT = float;
    static constexpr bool SHIFT = false;
    template <class Pol = LdStream> __device__ static T ld(const float *a) { return Pol::ld(a); }
    __device__ static void st(float *a, T v) { __stcs(a, v); }
};
template <> struct Store<__half> {
    using T = float;
    using PsiT = float;
    static constexpr bool SHIFT = true;
    template <class Pol = LdStream> __device__ static T ld(const __half *a) {
        return __half2float(__ushort_as_half(Pol::ld(reinterpret_cast<const unsigned short *>(a))));
    }
    __device__ static void st(__half *a, T v) {
        __stcs(reinterpret_cast<unsigned short *>(a), __half_as_ushort(__float2half_rn(v)));
    }
    // Stochastic rounding: uniform noise of +-1/2 FP16 ulp (at v's magnitude) added before
    // round-to-nearest, so the stored value is v in expectation.  r: 16 random bits.
    __device__ static float sr_dither(float v, unsigned r) {
        int e = (int)(__float_as_uint(v) & 0x7f800000u) - (10 << 23);    // 2^(exp - 10)
        e = e > ((127 - 24) << 23) ? e : ((127 - 24) << 23);            // subnormal halves: 2^-24
        const float ulp = __uint_as_float((unsigned)e);
        const float u = __uint_as_float(0x3f800000u | ((r & 0xffffu) << 7)) - 1.5f;   // [-1/2, 1/2)
        return fmaf(ulp, u, v);
    }
    __device__ static void st_sr(__half *a, T v, unsigned r) { st(a, sr_dither(v, r)); }
};

// Counter-based random bits for stochastic rounding: a 32-bit finaliser (murmur3 fmix32)
// of the cell index and the step counter, then one multiply-xorshift per direction.
__device__ __forceinline__ unsigned cell_hash(unsigned s, unsigned salt) {
    unsigned h = s * 0x9e3779b1u ^ (salt + 0x7f4a7c15u) * 0x85ebca6bu;
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
__device__ __forceinline__ unsigned dir_bits(unsigned h, int i) {
    unsigned r = (h ^ (0x9e3779b9u * (unsigned)(i + 1))) * 0xc2b2ae35u;
    return r ^ (r >> 15);
}

// Parameters in the arithmetic precision.
template <class T> __device__ __forceinline__ const Phys<T> &phys(const KParams &p);
template <> __device__ __forceinline__ const Phys<double> &phys<double>(const KParams &p) { return p.d; }
template <> __device__ __forceinline__ const Phys<float> &phys<float>(const KParams &p) { return p.f; }

// a * b + c: fused in FP32; in FP64 rounded after the product and after the sum (no
// contraction), which keeps the FP64 path's rounding close to a plain evaluation.
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return __dadd_rn(__dmul_rn(a, b), c); }
// a / b: the fast hardware reciprocal in FP32 (a few ulp), IEEE division in FP64.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

// ----------------------------------------------------------------- utilities
template <int I, int N> struct Unroll {
    template <class Fn> __device__ __forceinline__ static void run(Fn &&fn) {
        fn(std::integral_constant<int, I>{});
        Unroll<I + 1, N>::run(fn);
    }
};
template <int N> struct Unroll<N, N> {
    template <class Fn> __device__ __forceinline__ static void run(Fn &&) {}
};

// Neighbour coordinates with periodic wrap.
struct Nbr {
    int x[3], y[3], z[3];   // index 0: -1, 1: 0, 2: +1
};

__device__ __forceinline__ Nbr neighbours(const KParams &p, int x, int y, int z) {
    Nbr nb;
    nb.x[0] = x > 0 ? x - 1 : p.nx - 1;
    nb.x[1] = x;
    nb.x[2] = x < p.nx - 1 ? x + 1 : 0;
    nb.y[0] = y > 0 ? y - 1 : p.ny - 1;
    nb.y[1] = y;
    nb.y[2] = y < p.ny - 1 ? y + 1 : 0;
    nb.z[0] = z > 0 ? z - 1 : p.nz - 1;
    nb.z[1] = z;
    nb.z[2] = z < p.nz - 1 ? z + 1 : 0;
    return nb;
}

__device__ __forceinline__ long long cell_of(const KParams &p, int x, int y, int z) {
    return (long long)x + (long long)p.nx * ((long long)y + (long long)p.ny * z);
}

// Is x + d*c_i (d = +-1) outside the fluid rows?  Only y can hold walls.
__device__ __forceinline__ bool y_wall(const KParams &p, int y, int dy) {
    return p.wall_y && (y + dy < 0 || y + dy >= p.ny);
}

// Loads the Q pre-collision populations f_i (shift included) of cell (x, y, z): readout path.
template <class L, class S>
__device__ __forceinline__ void load_pops(const KParams &p, const S *__restrict__ A, int x, int y, int z,
                                          const Nbr &nb, long long s, bool odd, typename Store<S>::T *f) {
    using T = typename Store<S>::T;
    const T rref = phys<T>(p).rho_ref;
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int o = opp(i);
        T v;
        if (!odd) {
            v = Store<S>::ld(A + (long long)i * p.pstride + s);
        } else if (i != 0 && L::cy(i) != 0 && y_wall(p, y, -L::cy(i))) {
            v = Store<S>::ld(A + (long long)i * p.pstride + s);
        } else {
            // value streamed from x - c_i, stored in slot opp(i)
            const long long src = cell_of(p, nb.x[1 - L::cx(i)], nb.y[1 - L::cy(i)], nb.z[1 - L::cz(i)]);
            v = Store<S>::ld(A + (long long)o * p.pstride + src);
        }
        f[i] = Store<S>::SHIFT ? v + (T)L::w(i) * rref : v;
    });
}

// ------------------------------------------------------------------ the EOS
template <class T> __device__ __forceinline__ T eos_pressure(const KParams &p, T rho) {
    const Phys<T> &q = phys<T>(p);
    T pr;
    if (p.eos_kind == 0) {
        const T br = q.pr_b * rho;
        if (sizeof(T) == 4) {
            // one division: [rho RT D2 - a alpha rho^2 D1] / (D1 D2)
            const T d1 = (T)1 - br, d2 = (T)1 + br * ((T)2 - br);
            pr = fdiv(rho * mad(q.pr_RT, d2, -q.pr_aalpha * rho * d1), d1 * d2);
        } else {
            pr = rho * q.pr_RT / ((T)1 - br) - q.pr_aalpha * rho * rho / ((T)1 + (T)2 * br - br * br);
        }
    } else {
        // Eq. EOS with rho^2.5 = rho^2 sqrt(rho) etc.
        const T sr = sqrt(rho);
        const T rv = q.pe_rv, rl = q.pe_rl, sv = q.pe_sv;
        const T r2 = rho * rho;
        pr = q.pe_P * ((T)2 * r2 * rho + (rv - (T)2 * rl) * r2 - (T)3 * sv * r2 * sr + (T)2 * sv * rl * rho * sr +
                       sv * rl * rl * sr);
    }
    return q.p_scale * pr;
}

// psi of Eq. Interaction_Potential; raises the device flags on a domain error.
template <class T> __device__ __forceinline__ T psi_of(const KParams &p, T rho) {
    const Phys<T> &q = phys<T>(p);
    const T e = eos_pressure<T>(p, rho) - rho * (T)(1.0 / 3.0);
    const T arg = sizeof(T) == 4 ? (T)2 * e * q.inv_G : (T)2 * e / q.G;
    if (!(rho > (T)0) || !(rho < (T)INFINITY)) {
        atomicOr(p.flags, FLAG_NONFINITE);
        return (T)0;
    }
    if (!(arg >= (T)0)) {
        atomicOr(p.flags, FLAG_PSI_DOMAIN);
        return (T)0;
    }
    return sqrt(arg);
}

// -------------------------------------------------------------- force stencil
// Total force density at a cell from the padded psi field (pc = padded index): readout path.
template <class L, class T, class PsiT>
__device__ __forceinline__ void cell_force(const KParams &p, const PsiT *__restrict__ psi, long long pc, T F[3]) {
    const Phys<T> &q = phys<T>(p);
    const T psi0 = (T)__ldg(psi + pc);
    T m1[3] = {0, 0, 0};
    T m2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const long long sy = p.px, sz = (long long)p.px * p.py;
    Unroll<0, (L::Q - 1) / 2>::run([&](auto kc) {
        constexpr int i = 2 * decltype(kc)::value + 1;   // pair (i, i + 1), c_{i+1} = -c_i
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const long long off = cx + cy * sy + cz * sz;
        const T pa = (T)__ldg(psi + pc + off), pb = (T)__ldg(psi + pc - off);
        const T dif = pa - pb;                         // antisymmetric part: M1
        const T sym = pa + pb - (T)2 * psi0;           // symmetric part: M2 (sum_i w_i (cc - d/3) = 0)
        constexpr double w3 = 3.0 * L::w(i), w9 = 9.0 * L::w(i);
        constexpr int c[3] = {cx, cy, cz};
#pragma unroll
        for (int a = 0; a < L::D; ++a) {
            if (c[a] != 0) m1[a] = mad((T)(w3 * c[a]), dif, m1[a]);
#pragma unroll
            for (int b = a; b < L::D; ++b) {
                constexpr double third = 1.0 / 3.0;
                const double coef = w9 * (c[a] * c[b] - (a == b ? third : 0.0));
                if (coef != 0.0) m2[a][b] = mad((T)coef, sym, m2[a][b]);
            }
        }
    });
    T tr = 0;
#pragma unroll
    for (int a = 0; a < L::D; ++a) tr += m2[a][a];
    const T mG = -q.G * psi0, Ac = q.A_m1m2, Bt = q.B_m1tr * tr;
#pragma unroll
    for (int a = 0; a < L::D; ++a) {
        T m21 = 0;
#pragma unroll
        for (int b = 0; b < L::D; ++b) m21 = mad(a <= b ? m2[a][b] : m2[b][a], m1[b], m21);
        F[a] = mad(mG + Bt, m1[a], mad(Ac, m21, q.fext[a]));
    }
    if (L::D == 2) F[2] = 0;
}

// 1 / tau(rho) of Sec. VI (interpolation weight clamped to [0, 1]).
template <class T> __device__ __forceinline__ T omega_of(const KParams &p, T rho) {
    using R = typename ScalarOf<T>::type;
    const Phys<R> &q = phys<R>(p);
    if (!p.var_tau) return T(q.om_const);
    const T wgt = clamp01((rho - T(q.tau_rho_v)) * T(q.inv_drho_tau));
    return fdiv(T(1), mad(wgt, T(q.tau_l - q.tau_v), T(q.tau_v)));
}

// Padded psi index of interior cell (x, y, z).
__device__ __forceinline__ long long psi_index(const KParams &p, int x, int y, int z) {
    return p.psi_origin + x + (long long)p.px * ((long long)y + (long long)p.py * z);
}

}  // namespace plb
