// common.cuh -- shared device definitions of the RBSOG CUDA path (sm_103a).
//
// Device layout of a context (all systems concatenated):
//   per atom (original order): r, p, F (FP64 x3), q, mass (FP64), type, mol,
//     sys (int); binning products cell, rank (int), loc (cell-local coordinates,
//     float4/double4), su (fixed-point fractional coordinates + charge, uint4).
//   per cell (global index = cell0 of the system + local index, x fastest):
//     count, start; cell-sorted copies pos4 / posd, qt / aux, sidx.
//   pair work items (cell, 32-atom group), per system in [item0, item0 + item_cap).
//   per system: DevSys (box, box momenta, cell grid, normalizers, flags).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rbsog {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.283185307179586;
constexpr int kMaxGauss = 64;      // Gaussians of the split, M and M_energy
constexpr int kMaxP = 4096;        // batch size
constexpr int kCellCap = 2048;     // atoms per cell the kernels accept
constexpr int kChunk = 1024;       // atoms per chunk of the per-atom kernels
constexpr int kMolChunk = 32;      // molecules per block of the molecule kernel (small molecules)
constexpr int kMolChunkLarge = 16; // ... for systems of large molecules (a warp each)
constexpr int kSmallTerms = 24;    // terms of a molecule that one thread takes
constexpr int kMaxTypes = 16;
constexpr int kClus = 4;          // atoms per cluster of the FP32 pair kernel
constexpr double kFixScale = 4294967296.0;   // FP32 pair forces: 64-bit fixed point, units of 2^-32

// status flags written by kernels (bit mask in DevSys::flags)
enum : int {
    FLAG_BOX = 1,          // box edge below 3 cells of r_c
    FLAG_OVERFLOW = 2,     // a cell holds more than kCellCap atoms
    FLAG_NONFINITE = 4,
};

// Per-system device record.
struct DevSys {
    double L[3];          // box edges
    double ph[3];         // box momenta per coupling group (g/mol A/fs)
    double Mbox[3];       // box masses per group (<= 0: fixed)
    double V;
    double w[3];          // cell widths L / n
    double Sr, Snr;       // normalizers (eqs. Sr, Snr)
    double Lh[3];         // box after the first half drift (integrator)
    double Lp[3];         // box before the step (integrator)
    double sc1[3], sc2[3];   // drift scalings Lh / Lp and L / Lh of the current step
    double isc1[3], isc2[3]; // their inverses Lp / Lh and Lh / L
    double invL[3];          // 1 / L after the step
    int ncell[3];         // current cells per axis
    int ncap[3];          // allocated cells per axis
    int cell0;            // first global cell
    int ncell_cap_total;  // ncap[0]*ncap[1]*ncap[2]
    int atom0, n;
    int nD;               // distinct modes of the last evaluation
    int nacc_r, nacc_nr;
    int coupling;
    int flags;
    int item0, item_cap;  // pair-kernel work items: [item0, item0 + item_cap)
    int nitems;           // items of the current cell list
    int ntypes, lj0;      // LJ types of the system and its first entry in the context's LJ table
    int nmol, mol0;       // molecules of the system and its first global molecule index
    int act;              // 1: the slot holds a system that steps; 0: empty or finished
    int kc;               // FP32 build: sub-columns per cell axis of the in-cell atom order
    int steps_left;       // NPT steps before the system stops (-1: no limit)
    int rebuild;          // 1: this evaluation bins the atoms and rebuilds the pair lists
    int list_valid;       // 0: positions or box were set from the host since the last build
    int list_builds;      // pair-list builds so far
    double Lref[3];       // box at the last list build
    double thr2;          // squared displacement bound of the current step (lists with a skin)
    unsigned long long rng_id;   // second word of the Philox key
    unsigned long long step;     // Philox counter of the system's last force evaluation
    // triclinic cell (held fixed): h = [[L0, xy, xz], [0, L1, yz], [0, 0, L2]],
    // cell vectors as columns; all zero for an orthorhombic box
    double tilt[3];       // (xy, xz, yz)
    double tw[3];         // tilt per cell: xy / ncell[1], xz / ncell[2], yz / ncell[2]
    int tri;              // 1: some tilt is non-zero
};

// Atoms of a system that take part in the current step (0 for an empty or
// finished slot).
__host__ __device__ inline int live_n(const DevSys &d) { return d.act ? d.n : 0; }

// Per-distinct-mode data handed from the estimator to the force kernel.
struct ModeCoef {
    double a[3];          // alpha_d k_d: force on i is q_i a (rho_im cos - rho_re sin)
    double re, im;        // rho(k_d)
    int m[3];
    int pad;
};

// Philox4x64-10 (Salmon et al., SC'11), written from its published definition.
__host__ __device__ inline void philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
#ifdef __CUDA_ARCH__
        uint64_t hi0 = __umul64hi(M0, x0), lo0 = M0 * x0;
        uint64_t hi1 = __umul64hi(M1, x2), lo1 = M1 * x2;
#else
        unsigned __int128 p0 = (unsigned __int128)M0 * x0, p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
#endif
        uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// Philox counter purposes: counter = (step, purpose, index, 0), key = (seed, system).
enum : uint64_t { PUR_START = 1, PUR_PROPOSAL = 2, PUR_ACCEPT = 3, PUR_NR_IID = 4, PUR_ATOM = 5, PUR_BOX = 6 };

__host__ __device__ inline void draw4(uint64_t seed, uint64_t sys, uint64_t step, uint64_t purpose,
                                      uint64_t index, uint64_t out[4])
{
    const uint64_t ctr[4] = {step, purpose, index, 0};
    const uint64_t key[2] = {seed, sys};
    philox4x64(ctr, key, out);
}

// uniform in (0,1): ((x >> 12) + 1/2) 2^-52
__host__ __device__ inline double u01(uint64_t x)
{
    return ((double)(x >> 12) + 0.5) * 2.220446049250313e-16;
}

__device__ inline unsigned lane_id() { return threadIdx.x & 31u; }

__device__ inline double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ inline float warp_sumf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of an FP64 value (all threads get it).  smem >= 32 doubles.
__device__ inline double block_sum(double v, double *smem)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane_id() == 0) smem[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += smem[i];
    __syncthreads();
    return t;
}

// Block-wide sums of V FP64 values per thread (NT threads), written to
// out[0..V) (fixed order: deterministic).  FP64 arithmetic is slow on
// this GPU, so the sums run lane-parallel (each FP64 instruction adds for 32
// lanes) instead of as a shuffle tree.  smem: V * (NT + 1) + 4 V doubles;
// every thread of the block must call it.
template <int V, int NT>
__device__ inline void block_reduce_lanes(const double (&v)[V], double *smem, double *out)
{
    static_assert(NT % 4 == 0, "NT must be a multiple of 4");
    constexpr int G = 4, SEG = NT / G, ROW = NT + 1;
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < V; ++k) smem[k * ROW + t] = v[k];
    __syncthreads();
    double *s2 = smem + V * ROW;
    for (int idx = t; idx < V * G; idx += NT) {
        const int k = idx / G, g = idx % G;
        const double *p = smem + k * ROW + g * SEG;
        double a = 0.0;
        for (int i = 0; i < SEG; ++i) a += p[i];
        s2[k * G + g] = a;
    }
    __syncthreads();
    for (int k = t; k < V; k += NT) out[k] = (s2[k * G] + s2[k * G + 1]) + (s2[k * G + 2] + s2[k * G + 3]);
}

// Perpendicular width of the cell of d along axis a (the distance between
// the two faces the a-th cell vector joins): V / |b x c| etc.; L_a when the
// cell is orthorhombic.
__host__ __device__ inline double perp_width(const double L[3], const double t[3], int a)
{
    const double xy = t[0], xz = t[1], yz = t[2];
    if (a == 2) return L[2];
    if (a == 1) return L[1] * L[2] / sqrt(L[2] * L[2] + yz * yz);
    const double b0 = L[1] * L[2], b1 = xy * L[2], b2 = xy * yz - L[1] * xz;
    return L[0] * L[1] * L[2] / sqrt(b0 * b0 + b1 * b1 + b2 * b2);
}

// Cell grid of one axis for box edge L (cells of r_c / sub, at least
// 2 sub + 1 and at most the slot's capacity ncap): sets *bad when the box is
// too small, not finite or beyond the allocated grid.
__device__ __forceinline__ int axis_cells(double L, int sub, double rc, int ncap, bool *bad)
{
    const int minc = 2 * sub + 1;
    const double x = floor(__ddiv_rn(__dmul_rn(L, (double)sub), rc));
    if (!(L > 0.0) || !(x < 1e9) || x < (double)minc) *bad = true;
    int n = (x < 1e9 && x >= (double)minc) ? (int)x : minc;
    if (n > ncap) n = ncap;
    return n;
}

// Fractional coordinates s = h^{-1} x for the upper-triangular h of d, by back
// substitution; an orthorhombic box takes s_a = x_a / L_a, three independent
// divisions (the substitution chains them, and FP64 divisions are long
// sequences on this part's FP64 pipe: chained, they tripled the latency of
// the binning kernels).
__device__ __forceinline__ void frac_of(const DevSys &d, const double x[3], double s[3])
{
    if (!d.tri) {
#pragma unroll
        for (int a = 0; a < 3; ++a) s[a] = __ddiv_rn(x[a], d.L[a]);
        return;
    }
    s[2] = __ddiv_rn(x[2], d.L[2]);
    s[1] = __ddiv_rn(__dsub_rn(x[1], __dmul_rn(d.tilt[2], s[2])), d.L[1]);
    s[0] = __ddiv_rn(__dsub_rn(__dsub_rn(x[0], __dmul_rn(d.tilt[0], s[1])), __dmul_rn(d.tilt[1], s[2])), d.L[0]);
}

// x - h n for an integer vector n (a lattice translation of the cell of d)
__device__ __forceinline__ void sub_lattice(const DevSys &d, const double n[3], double x[3])
{
    x[0] -= d.L[0] * n[0] + d.tilt[0] * n[1] + d.tilt[1] * n[2];
    x[1] -= d.L[1] * n[1] + d.tilt[2] * n[2];
    x[2] -= d.L[2] * n[2];
}

// Minimum image of a difference vector in the tilted cell of d: the image
// whose fractional components lie in [-1/2, 1/2].  For two atoms within r_c
// that is the image within r_c (every perpendicular width of the cell is
// above 2 r_c, as the cell grid requires).
__device__ __forceinline__ void min_image_tri(const DevSys &d, double x[3])
{
    double s[3], n[3];
    frac_of(d, x, s);
#pragma unroll
    for (int a = 0; a < 3; ++a) n[a] = rint(s[a]);
    sub_lattice(d, n, x);
}

// k = 2 pi h^{-T} m for the cell of d (h^T k = 2 pi m, forward substitution)
__device__ __forceinline__ void kvec_of(const DevSys &d, const int m[3], double k[3])
{
    k[0] = (kTwoPi * (double)m[0]) / d.L[0];
    k[1] = (kTwoPi * (double)m[1] - d.tilt[0] * k[0]) / d.L[1];
    k[2] = (kTwoPi * (double)m[2] - d.tilt[1] * k[0] - d.tilt[2] * k[1]) / d.L[2];
}

// Bin atom i of system d at position x (wrapped into [0, L)): its cell, its
// rank there by a warp-aggregated atomic on count (act: the lanes of the warp
// that bin an atom), cell-local coordinates and fixed-point fractional
// coordinates.
__device__ __forceinline__ void bin_atom(const DevSys &d, int i, const double x[3], double qi, int moli,
                                         unsigned act, int *__restrict__ cell, int *__restrict__ rank,
                                         int *__restrict__ count, float4 *__restrict__ locf,
                                         double4 *__restrict__ locd, uint4 *__restrict__ su, int precision, bool fast = false)
{
    int c[3];
    double sf[3], xl[3];
    if (fast && !d.tri) {
        // NPT steps: s = x (1/L), the reciprocal of the step's box half-step
        // (one FP64 multiply instead of an IEEE division; the cell of an atom
        // within an ulp of a cell face may differ from the division's, which
        // any consistent binning allows)
#pragma unroll
        for (int a = 0; a < 3; ++a) sf[a] = x[a] * d.invL[a];
    } else {
        frac_of(d, x, sf);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double L = d.L[a];
        double s = sf[a];
        s = __dsub_rn(s, floor(s));
        if (s >= 1.0) s = 0.0;
        int n = d.ncell[a];
        int k = (int)floor(__dmul_rn(s, (double)n));
        if (k > n - 1) k = n - 1;
        if (!(k >= 0)) k = 0;        // non-finite coordinates (flagged by the step checks)
        c[a] = k;
        sf[a] = s;
        xl[a] = s * L - k * d.w[a];
    }
    if (d.tri) {
        // cell-local Cartesian coordinates h (s - c / n): the tilt terms
        xl[0] += (d.tilt[0] * sf[1] - c[1] * d.tw[0]) + (d.tilt[1] * sf[2] - c[2] * d.tw[1]);
        xl[1] += d.tilt[2] * sf[2] - c[2] * d.tw[2];
    }
    const int gc = d.cell0 + c[0] + d.ncell[0] * (c[1] + d.ncell[1] * c[2]);
    cell[i] = gc;
    // warp-aggregated atomic: one atomicAdd per distinct cell in the warp
    const unsigned peers = __match_any_sync(act, gc);
    const int leader = __ffs(peers) - 1;
    const unsigned lane = threadIdx.x & 31u;
    int base = 0;
    if ((int)lane == leader) base = atomicAdd(&count[gc], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    rank[i] = base + __popc(peers & ((1u << lane) - 1u));
    if (precision == 1) {
        locf[i] = make_float4((float)xl[0], (float)xl[1], (float)xl[2], __int_as_float(moli));
        su[i] = make_uint4(__double2uint_rz(sf[0] * 4294967296.0), __double2uint_rz(sf[1] * 4294967296.0),
                           __double2uint_rz(sf[2] * 4294967296.0), __float_as_uint((float)qi));
    } else {
        locd[i] = make_double4(xl[0], xl[1], xl[2], qi);
    }
}

}  // namespace rbsog
