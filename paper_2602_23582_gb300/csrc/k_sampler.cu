// k_sampler.cu -- Fourier-mode sampling for the random batch (paper sec. 3.2,
// App. D) and the normalizers S^r, S^nr (eqs. Sr, Snr).  One block per
// system.  Built with -fmad=false: every accept/reject and rounding decision
// is made with the same IEEE operations, in the same order, as the CPU oracle,
// so sampled mode indices agree bit for bit (barring ties within a rounding
// error of libm vs CUDA transcendentals).
//
// Steps (orthorhombic h, k = 2 pi m / L):
//  1. 1D lattice sums per Gaussian l and axis a (warp-parallel, FP64):
//     S_n = sum_m m^n e^{-a m^2}, a = (pi s~_l / L_a)^2, |m| <= ceil(sqrt(46/a)) + 2;
//     T0 = S0, T2 = (2pi/L)^2 S2, T4 = (2pi/L)^4 S4.  H^r_l and H^nr_l are sums
//     of products of these (e^{-s~^2 k^2/4} factorises over the axes).
//  2. exact draws from P^r (mixture over (l, axis) with weights c_l T2_a T0 T0)
//     or P^nr (six components per l), by warp-parallel inverse CDF scans.
//  3. radial MH chain (App. D): the proposal m* = round(L u), u ~ N(0, 1/(2 pi^2
//     s~0^2)), depends on no state, so the weights w(m*) = P^r(m*) / q(m*)
//     (q from eq. proposal, factorised with erf/erfc) of all P proposals are
//     evaluated in parallel; one thread then runs the accept test
//     u_t w(x) < w(m*), i.e. u_t < P^r(m*) q(x) / (P^r(x) q(m*)) (eq. acc_Gaussian).
//  4. recalibration chain (sec. 3.2): proposals are the radial samples;
//     accept iff u'_t g(y) < g(x_t) with g = P^nr / P^r.
//  5. distinct modes of the union, lexicographic order, multiplicities.
//
// A tilted cell (DevSys::tri, h = [[L0, xy, xz], [0, L1, yz], [0, 0, L2]],
// held fixed): k = 2 pi h^{-T} m; the lattice sums over Z^3 are made once per
// cell (k_tri_gy, k_tri_reduce); the proposal is m* = round(h^T u) and its
// mass q(m*) the probability that h^T u lies in the unit cube around m*: an
// erf difference in u_2 given (u_0, u_1), Gauss-Legendre quadrature over
// (u_0, u_1); the chain's start is an exact draw of P^r: component (l, a)
// with weight c_l sum_m k_a^2 e_l, then m_0, m_1 given m_0 and m_2 given
// (m_0, m_1) by inverse CDF over m = 0, 1, -1, 2, ... (tables for m_0 and m_1).
#include "internal.h"

namespace rbsog {

namespace {

struct Shared {
    double T0[kMaxGauss][3], T2[kMaxGauss][3], T4[kMaxGauss][3];
    double Hr[kMaxGauss], Hnr[kMaxGauss];
    double Sr, Snr;
    double L[3];
    int sel_l[8], sel_c[8];   // per warp (256-thread blocks)
    int nd;
};

// terms beyond |m| = ceil(sqrt(46 / a)) + 2 are below e^-46 of the largest;
// capped so that a non-finite box (flagged, step discarded) cannot run away
__device__ int axis_mmax(double a)
{
    const double x = ceil(sqrt(46.0 / a));
    return (x < 65536.0 ? (int)x : 65536) + 2;
}

// unnormalised targets (eqs. samplingP, samplingPnr)
__device__ void targets(const SamplerArgs &sa, const double L[3], const int m[3], double &pr, double &pnr)
{
    double kx = (kTwoPi * (double)m[0]) / L[0];
    double ky = (kTwoPi * (double)m[1]) / L[1];
    double kz = (kTwoPi * (double)m[2]) / L[2];
    double k2 = kx * kx + ky * ky + kz * kz;
    double a = 0.0, b = 0.0;
    for (int l = 0; l < sa.M; ++l) {
        double e = exp(-(sa.st2q[l] * k2));
        a += sa.cr[l] * e;
        b += sa.cn[l] * e;
    }
    pr = k2 * a;
    pnr = (k2 * k2) * b;
}

__device__ double q1d(int m, double L, double st0)
{
    double c = kPi * st0 / L;
    int am = m < 0 ? -m : m;
    if (am == 0) return erf(c * 0.5);
    double lo = c * ((double)am - 0.5), hi = c * ((double)am + 0.5);
    return 0.5 * (erfc(lo) - erfc(hi));
}

__device__ double qprop(const SamplerArgs &sa, const double L[3], const int m[3])
{
    return q1d(m[0], L[0], sa.st[0]) * q1d(m[1], L[1], sa.st[0]) * q1d(m[2], L[2], sa.st[0]);
}

// one coordinate from m^{2n} e^{-a m^2}: inverse CDF over m = 0, 1, -1, 2, -2, ...
// (warp-parallel prefix sums; returns the same m on every lane)
__device__ int draw_axis_warp(double u, double stl, double L, int n, double total)
{
    const int lane = lane_id();
    double c = kPi * stl / L, a = c * c;
    int mm = axis_mmax(a);
    double target = u * total, cum = 0.0;
    const int kmax = 2 * mm;
    for (int k0 = 0; k0 <= kmax; k0 += 32) {
        int k = k0 + lane;
        int m = (k == 0) ? 0 : ((k & 1) ? (k + 1) / 2 : -(k / 2));
        double m2 = (double)m * (double)m;
        double wgt = 0.0;
        if (k <= kmax) {
            wgt = exp(-(a * m2));
            if (n >= 1) wgt *= m2;
            if (n >= 2) wgt *= m2;
        }
        double incl = wgt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            double t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        unsigned hit = __ballot_sync(0xffffffffu, k <= kmax && cum + incl > target);
        if (hit) return __shfl_sync(0xffffffffu, m, __ffs(hit) - 1);
        cum += __shfl_sync(0xffffffffu, incl, 31);
    }
    int k = kmax;
    return (k == 0) ? 0 : ((k & 1) ? (k + 1) / 2 : -(k / 2));
}

__device__ double axis_total(const Shared &sh, int l, int a, int n)
{
    double g = kTwoPi / sh.L[a];
    if (n == 0) return sh.T0[l][a];
    if (n == 1) return sh.T2[l][a] / (g * g);
    return sh.T4[l][a] / (g * g * g * g);
}

// exact draw from P^r (nr = false) or P^nr (nr = true) by one warp
__device__ void exact_draw_warp(const SamplerArgs &sa, Shared &sh, const uint64_t wds[4], bool nr, int m[3])
{
    const int lane = lane_id();
    if (lane == 0) {
        double tot = 0.0;
        for (int l = 0; l < sa.M; ++l) tot += nr ? sh.Hnr[l] : sh.Hr[l];
        double target = u01(wds[0]) * tot, cum = 0.0;
        int lsel = sa.M - 1, csel = nr ? 5 : 2;
        bool done = false;
        for (int l = 0; l < sa.M && !done; ++l) {
            const double *T0 = sh.T0[l], *T2 = sh.T2[l], *T4 = sh.T4[l];
            double comp[6];
            int nc;
            if (!nr) {
                comp[0] = sa.cr[l] * T2[0] * T0[1] * T0[2];
                comp[1] = sa.cr[l] * T0[0] * T2[1] * T0[2];
                comp[2] = sa.cr[l] * T0[0] * T0[1] * T2[2];
                nc = 3;
            } else {
                comp[0] = sa.cn[l] * T4[0] * T0[1] * T0[2];
                comp[1] = sa.cn[l] * T0[0] * T4[1] * T0[2];
                comp[2] = sa.cn[l] * T0[0] * T0[1] * T4[2];
                comp[3] = 2.0 * sa.cn[l] * T2[0] * T2[1] * T0[2];
                comp[4] = 2.0 * sa.cn[l] * T2[0] * T0[1] * T2[2];
                comp[5] = 2.0 * sa.cn[l] * T0[0] * T2[1] * T2[2];
                nc = 6;
            }
            for (int t = 0; t < nc; ++t) {
                cum += comp[t];
                if (cum > target) { lsel = l; csel = t; done = true; break; }
            }
        }
        sh.sel_l[threadIdx.x >> 5] = lsel;
        sh.sel_c[threadIdx.x >> 5] = csel;
    }
    __syncwarp();
    const int lsel = sh.sel_l[threadIdx.x >> 5], csel = sh.sel_c[threadIdx.x >> 5];
    __syncwarp();
    static const int pr_pw[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    static const int pn_pw[6][3] = {{2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
    for (int a = 0; a < 3; ++a) {
        int n = nr ? pn_pw[csel][a] : pr_pw[csel][a];
        m[a] = draw_axis_warp(u01(wds[1 + a]), sa.st[lsel], sh.L[a], n, axis_total(sh, lsel, a, n));
    }
}

__device__ inline uint64_t mode_key(const int m[3])
{
    const uint64_t B = 1u << 20;
    return ((uint64_t)(m[0] + B) << 42) | ((uint64_t)(m[1] + B) << 21) | (uint64_t)(m[2] + B);
}

__device__ inline void key_mode(uint64_t k, int m[3])
{
    const int B = 1 << 20;
    m[0] = (int)((k >> 42) & 0x1fffff) - B;
    m[1] = (int)((k >> 21) & 0x1fffff) - B;
    m[2] = (int)(k & 0x1fffff) - B;
}

}  // namespace

// Step 1 on its own grid: one warp per (system, Gaussian l, axis).
__global__ void __launch_bounds__(32)
k_samp_sums(const DevSys *sys, const SamplerArgs sa, SampScratch *ss)
{
    const int s = blockIdx.x, idx = blockIdx.y, lane = lane_id();
    const DevSys &d = sys[s];
    if ((d.flags & FLAG_BOX) || live_n(d) == 0 || idx >= 3 * sa.M || d.tri) return;   // tilted: k_tri_*
    const int l = idx / 3, ax = idx % 3;
    const double L = d.L[ax];
    double c = kPi * sa.st[l] / L, a = c * c;
    int mm = axis_mmax(a);
    double s0 = 0.0, s2 = 0.0, s4 = 0.0;
    for (int m = -mm + lane; m <= mm; m += 32) {
        double m2 = (double)m * (double)m;
        double e = exp(-(a * m2));
        s0 += e; s2 += m2 * e; s4 += m2 * m2 * e;
    }
    s0 = warp_sum(s0); s2 = warp_sum(s2); s4 = warp_sum(s4);
    if (lane == 0) {
        double g = kTwoPi / L;
        ss[s].T[0][l][ax] = s0;
        ss[s].T[1][l][ax] = g * g * s2;
        ss[s].T[2][l][ax] = g * g * g * g * s4;
    }
}

// Shared copy of the lattice sums and H^r_l, H^nr_l (each lane l forms its
// Gaussian's terms; the sums over l run in order on every lane).
__device__ void load_sums(const SamplerArgs &sa, const SampScratch &sc, const double L[3], Shared &sh,
                          double &sr, double &snr)
{
    const int lane = lane_id();
    for (int k = lane; k < 3 * sa.M; k += 32) {
        const int l = k / 3, ax = k % 3;
        sh.T0[l][ax] = sc.T[0][l][ax];
        sh.T2[l][ax] = sc.T[1][l][ax];
        sh.T4[l][ax] = sc.T[2][l][ax];
    }
    if (lane < 3) sh.L[lane] = L[lane];
    __syncwarp();
    for (int l = lane; l < sa.M; l += 32) {
        const double *T0 = sh.T0[l], *T2 = sh.T2[l], *T4 = sh.T4[l];
        sh.Hr[l] = sa.cr[l] * (T2[0] * T0[1] * T0[2] + T0[0] * T2[1] * T0[2] + T0[0] * T0[1] * T2[2]);
        sh.Hnr[l] = sa.cn[l] * (T4[0] * T0[1] * T0[2] + T0[0] * T4[1] * T0[2] + T0[0] * T0[1] * T4[2]
                                + 2.0 * (T2[0] * T2[1] * T0[2] + T2[0] * T0[1] * T2[2] + T0[0] * T2[1] * T2[2]));
    }
    __syncwarp();
    sr = 0.0;
    snr = 0.0;
    for (int l = 0; l < sa.M; ++l) {
        sr += sh.Hr[l];
        snr += sh.Hnr[l];
    }
}

// P^r and P^nr (targets) for one mode by one warp: lane l forms the l-th
// exponential, the sums over l run in order as in targets().
__device__ void targets_warp(const SamplerArgs &sa, const double L[3], const int m[3], double &pr, double &pnr)
{
    const int lane = lane_id();
    double kx = (kTwoPi * (double)m[0]) / L[0];
    double ky = (kTwoPi * (double)m[1]) / L[1];
    double kz = (kTwoPi * (double)m[2]) / L[2];
    double k2 = kx * kx + ky * ky + kz * kz;
    double a = 0.0, b = 0.0;
    for (int l0 = 0; l0 < sa.M; l0 += 32) {
        const int l = l0 + lane;
        const double e = l < sa.M ? exp(-(sa.st2q[l] * k2)) : 0.0;
        const int nl = min(32, sa.M - l0);
        for (int u = 0; u < nl; ++u) {
            const double eu = __shfl_sync(0xffffffffu, e, u);
            a += sa.cr[l0 + u] * eu;
            b += sa.cn[l0 + u] * eu;
        }
    }
    pr = k2 * a;
    pnr = (k2 * k2) * b;
}

// q(m*) of eq. proposal by one warp: lane a forms the factor of axis a.
__device__ double qprop_warp(const SamplerArgs &sa, const double L[3], const int m[3])
{
    const int lane = lane_id();
    const int ax = lane < 3 ? lane : 0;
    const double q = q1d(m[ax], L[ax], sa.st[0]);
    const double q0 = __shfl_sync(0xffffffffu, q, 0), q1 = __shfl_sync(0xffffffffu, q, 1),
                 q2 = __shfl_sync(0xffffffffu, q, 2);
    return q0 * q1 * q2;
}

// ---- tilted cell ----------------------------------------------------------

__device__ inline int walk_m(int k) { return (k == 0) ? 0 : ((k & 1) ? (k + 1) / 2 : -(k / 2)); }

// P^r and P^nr (targets) of one mode in the tilted cell of d, by one warp
__device__ void targets_tri_warp(const SamplerArgs &sa, const DevSys &d, const int m[3], double &pr, double &pnr)
{
    const int lane = lane_id();
    double k[3];
    kvec_of(d, m, k);
    const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    double a = 0.0, b = 0.0;
    for (int l0 = 0; l0 < sa.M; l0 += 32) {
        const int l = l0 + lane;
        const double e = l < sa.M ? exp(-(sa.st2q[l] * k2)) : 0.0;
        const int nl = min(32, sa.M - l0);
        for (int u = 0; u < nl; ++u) {
            const double eu = __shfl_sync(0xffffffffu, e, u);
            a += sa.cr[l0 + u] * eu;
            b += sa.cn[l0 + u] * eu;
        }
    }
    pr = k2 * a;
    pnr = (k2 * k2) * b;
}

// P(lo <= u <= hi) for u ~ N(0, sig^2), without cancellation in the tails
__device__ double normal_interval(double lo, double hi, double sig)
{
    const double x = lo / (sqrt(2.0) * sig), y = hi / (sqrt(2.0) * sig);
    if (x >= 0.0) return 0.5 * (erfc(x) - erfc(y));
    if (y <= 0.0) return 0.5 * (erfc(-y) - erfc(-x));
    return 0.5 * (erf(y) - erf(x));
}

// q(m*) of eq. proposal in the tilted cell of d, by one warp: (h^T u)_0 =
// L0 u_0, (h^T u)_1 = xy u_0 + L1 u_1, (h^T u)_2 = xz u_0 + yz u_1 + L2 u_2;
// the u_2 interval in closed form, kGL x kGL Gauss-Legendre nodes over u_0
// and u_1 (one node pair per lane and pass)
__device__ double qprop_tri_warp(const SamplerArgs &sa, const DevSys &d, const int m[3])
{
    const int lane = lane_id();
    const double sig = sa.sig_u, nrm = 1.0 / (sqrt(2.0 * kPi) * sig), i2s2 = 1.0 / (2.0 * sig * sig);
    const double A0 = ((double)m[0] - 0.5) / d.L[0], B0 = ((double)m[0] + 0.5) / d.L[0];
    const double c0 = 0.5 * (A0 + B0), h0 = 0.5 * (B0 - A0);
    double acc = 0.0;
    for (int p = lane; p < kGL * kGL; p += 32) {
        const int i = p / kGL, j = p % kGL;
        const double u0 = c0 + h0 * sa.glx[i];
        const double A1 = ((double)m[1] - 0.5 - d.tilt[0] * u0) / d.L[1];
        const double B1 = ((double)m[1] + 0.5 - d.tilt[0] * u0) / d.L[1];
        const double u1 = 0.5 * (A1 + B1) + 0.5 * (B1 - A1) * sa.glx[j];
        const double c = d.tilt[1] * u0 + d.tilt[2] * u1;
        const double pz = normal_interval(((double)m[2] - 0.5 - c) / d.L[2], ((double)m[2] + 0.5 - c) / d.L[2], sig);
        acc += (sa.glw[i] * nrm * exp(-u0 * u0 * i2s2)) * (0.5 * (B1 - A1)) * (sa.glw[j] * nrm * exp(-u1 * u1 * i2s2)) * pz;
    }
    return warp_sum(acc) * h0;
}

// inverse CDF over m = 0, 1, -1, ... of tab[m + mm] (|m| <= mm), one warp
__device__ int walk_table_warp(double target, const double *__restrict__ tab, int mm)
{
    const int lane = lane_id();
    double cum = 0.0;
    const int kmax = 2 * mm;
    for (int k0 = 0; k0 <= kmax; k0 += 32) {
        const int k = k0 + lane;
        const int m = walk_m(k);
        double incl = k <= kmax ? tab[m + mm] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, k <= kmax && cum + incl > target);
        if (hit) return __shfl_sync(0xffffffffu, m, __ffs(hit) - 1);
        cum += __shfl_sync(0xffffffffu, incl, 31);
    }
    return walk_m(kmax);
}

// exact draw from P^r in the tilted cell of d, one warp (same on every lane)
__device__ void exact_draw_tri_warp(const SamplerArgs &sa, const DevSys &d, const SampScratch &sc,
                                    const uint64_t wds[4], int m[3])
{
    const int lane = lane_id();
    int sel = 0;
    if (lane == 0) {
        double tot = 0.0;
        for (int l = 0; l < sa.M; ++l) tot += sc.tHr[l];
        const double target = u01(wds[0]) * tot;
        double cum = 0.0;
        int lsel = sa.M - 1, asel = 2;
        bool done = false;
        for (int l = 0; l < sa.M && !done; ++l)
            for (int a = 0; a < 3; ++a) {
                cum += sa.cr[l] * sc.tS[l][a];
                if (cum > target) { lsel = l; asel = a; done = true; break; }
            }
        sel = 3 * lsel + asel;
    }
    sel = __shfl_sync(0xffffffffu, sel, 0);
    const int l = sel / 3, a = sel % 3;
    const int mm0 = sc.tmm[0], mm1 = sc.tmm[1], mm2 = sc.tmm[2];
    const size_t nx = 2 * mm0 + 1, ny = 2 * mm1 + 1;
    const double *Gy = sa.tri_tab + sc.tab0;
    const double *Gx = Gy + (size_t)sa.M * 3 * nx * ny;
    m[0] = walk_table_warp(u01(wds[1]) * sc.tS[l][a], Gx + (size_t)sel * nx, mm0);
    const size_t ix = (size_t)(m[0] + mm0);
    m[1] = walk_table_warp(u01(wds[2]) * Gx[(size_t)sel * nx + ix], Gy + ((size_t)sel * nx + ix) * ny, mm1);
    const size_t iy = (size_t)(m[1] + mm1);
    // m_2 given (m_0, m_1): weights k_a^2 e_l formed in walk order
    const double target = u01(wds[3]) * Gy[((size_t)sel * nx + ix) * ny + iy];
    double cum = 0.0;
    const int kmax = 2 * mm2;
    for (int k0 = 0; k0 <= kmax; k0 += 32) {
        const int k = k0 + lane;
        const int mz = walk_m(k);
        double incl = 0.0;
        if (k <= kmax) {
            const int mk[3] = {m[0], m[1], mz};
            double kv[3];
            kvec_of(d, mk, kv);
            const double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
            incl = kv[a] * kv[a] * exp(-(sa.st2q[l] * k2));
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, k <= kmax && cum + incl > target);
        if (hit) { m[2] = __shfl_sync(0xffffffffu, mz, __ffs(hit) - 1); return; }
        cum += __shfl_sync(0xffffffffu, incl, 31);
    }
    m[2] = walk_m(kmax);
}

// Steps 2-3 of the paper MH sampler on their own grid: block (s, t) is one
// warp; t < P evaluates proposal t (its three normals, its target and
// proposal masses lane-parallel), t = P draws the chain's start state exactly.
// Every value is formed by the same operations, in the same order, as the
// one-thread code of the CPU oracle.
__global__ void __launch_bounds__(32)
k_samp_prop(const DevSys *sys, const SamplerArgs sa, int adv, SampScratch *ss, int4 *__restrict__ pm,
            double *__restrict__ pw, double *__restrict__ pg, double *__restrict__ pu, double *__restrict__ pun)
{
    __shared__ Shared sh;
    const int s = blockIdx.x, t = blockIdx.y, lane = lane_id();
    const DevSys &d = sys[s];
    if ((d.flags & FLAG_BOX) || live_n(d) == 0) return;
    const uint64_t step = d.step + (uint64_t)adv;
    const int P = sa.P;
    const double L[3] = {d.L[0], d.L[1], d.L[2]};
    uint64_t wds[4];
    if (d.tri) return;                        // tilted cells: k_samp_prop_tri
    if (t == P) {
        double sr, snr;
        load_sums(sa, ss[s], L, sh, sr, snr);
        draw4(sa.seed, d.rng_id, step, PUR_START, 0, wds);
        int m[3];
        exact_draw_warp(sa, sh, wds, false, m);
        double pr, pnr;
        targets_warp(sa, L, m, pr, pnr);
        const double q = qprop_warp(sa, L, m);
        if (lane == 0) {
            SampScratch &sc = ss[s];
            sc.start_m[0] = m[0]; sc.start_m[1] = m[1]; sc.start_m[2] = m[2];
            sc.start_w = pr / q;
            sc.start_g = pnr / pr;
        }
        return;
    }
    draw4(sa.seed, d.rng_id, step, PUR_PROPOSAL, (uint64_t)t, wds);
    // z_0, z_1 from the first Box-Muller pair, z_2 from the second: lane a forms z_a
    double z = 0.0;
    if (lane < 3) {
        const double u1 = u01(lane < 2 ? wds[0] : wds[2]), u2 = u01(lane < 2 ? wds[1] : wds[3]);
        const double rr = sqrt(-2.0 * log(u1)), ang = kTwoPi * u2;
        z = rr * (lane == 1 ? sin(ang) : cos(ang));
    }
    const int ma = lane < 3 ? (int)floor(L[lane] * (z * sa.sig_u) + 0.5) : 0;
    int m[3];
    m[0] = __shfl_sync(0xffffffffu, ma, 0);
    m[1] = __shfl_sync(0xffffffffu, ma, 1);
    m[2] = __shfl_sync(0xffffffffu, ma, 2);
    double w = 0.0, g = 0.0;
    if (m[0] || m[1] || m[2]) {
        double pr, pnr;
        targets_warp(sa, L, m, pr, pnr);
        const double q = qprop_warp(sa, L, m);
        w = pr / q;
        g = pnr / pr;
    }
    if (lane == 0) {
        const size_t k = (size_t)s * P + t;
        pm[k] = make_int4(m[0], m[1], m[2], 0);
        pw[k] = w;
        pg[k] = g;
        draw4(sa.seed, d.rng_id, step, PUR_ACCEPT, (uint64_t)t, wds);
        pu[k] = u01(wds[0]);
        pun[k] = u01(wds[1]);
    }
}

// Steps 2-3 for the tilted cells (DevSys::tri), a kernel of its own so that
// the orthorhombic one keeps its code: block (s, t) as in k_samp_prop.
__global__ void __launch_bounds__(32)
k_samp_prop_tri(const DevSys *sys, const SamplerArgs sa, int adv, SampScratch *ss, int4 *__restrict__ pm,
                double *__restrict__ pw, double *__restrict__ pg, double *__restrict__ pu, double *__restrict__ pun)
{
    const int s = blockIdx.x, t = blockIdx.y, lane = lane_id();
    const DevSys &d = sys[s];
    if ((d.flags & FLAG_BOX) || live_n(d) == 0 || !d.tri) return;
    const uint64_t step = d.step + (uint64_t)adv;
    const int P = sa.P;
    uint64_t wds[4];
    int m[3];
    double w = 0.0, g = 0.0;
    if (t == P) {
        draw4(sa.seed, d.rng_id, step, PUR_START, 0, wds);
        exact_draw_tri_warp(sa, d, ss[s], wds, m);
    } else {
        draw4(sa.seed, d.rng_id, step, PUR_PROPOSAL, (uint64_t)t, wds);
        double z = 0.0;
        if (lane < 3) {
            const double u1 = u01(lane < 2 ? wds[0] : wds[2]), u2 = u01(lane < 2 ? wds[1] : wds[3]);
            const double rr = sqrt(-2.0 * log(u1)), ang = kTwoPi * u2;
            z = rr * (lane == 1 ? sin(ang) : cos(ang));
        }
        const double z0 = __shfl_sync(0xffffffffu, z, 0), z1 = __shfl_sync(0xffffffffu, z, 1),
                     z2 = __shfl_sync(0xffffffffu, z, 2);
        // gamma = h^T (sigma_u z)
        const double g0 = d.L[0] * (z0 * sa.sig_u);
        const double g1 = d.L[1] * (z1 * sa.sig_u) + d.tilt[0] * (z0 * sa.sig_u);
        const double g2 = d.L[2] * (z2 * sa.sig_u) + (d.tilt[1] * (z0 * sa.sig_u) + d.tilt[2] * (z1 * sa.sig_u));
        m[0] = (int)floor(g0 + 0.5);
        m[1] = (int)floor(g1 + 0.5);
        m[2] = (int)floor(g2 + 0.5);
    }
    if (t == P || m[0] || m[1] || m[2]) {
        double pr, pnr;
        targets_tri_warp(sa, d, m, pr, pnr);
        const double q = qprop_tri_warp(sa, d, m);
        w = pr / q;
        g = pnr / pr;
    }
    if (lane == 0) {
        if (t == P) {
            SampScratch &sc = ss[s];
            sc.start_m[0] = m[0]; sc.start_m[1] = m[1]; sc.start_m[2] = m[2];
            sc.start_w = w;
            sc.start_g = g;
        } else {
            const size_t k = (size_t)s * P + t;
            pm[k] = make_int4(m[0], m[1], m[2], 0);
            pw[k] = w;
            pg[k] = g;
            draw4(sa.seed, d.rng_id, step, PUR_ACCEPT, (uint64_t)t, wds);
            pu[k] = u01(wds[0]);
            pun[k] = u01(wds[1]);
        }
    }
    return;
}

// scratch per system: [P] proposal modes (int4) + w, g, u_r, u_nr (double)
__global__ void __launch_bounds__(256)
k_sampler(DevSys *sys, const SamplerArgs sa, int adv, int *__restrict__ mr_out, int *__restrict__ mnr_out,
          int *__restrict__ D_out, int *__restrict__ cr_out, int *__restrict__ cnr_out,
          int4 *__restrict__ pm, double *__restrict__ pw, double *__restrict__ pg,
          double *__restrict__ pu, double *__restrict__ pun, const SampScratch *__restrict__ ss, int Dcap)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    uint64_t *keys = reinterpret_cast<uint64_t *>(dyn);         // [2 * P2]
    __shared__ Shared sh;
    __shared__ int start_m[3], nrstart_m[3];
    __shared__ double start_w, start_g, nrstart_g;
    __shared__ int cnt_r, cnt_nr;
    __shared__ int scan_w[8];
    const int s = blockIdx.x;
    DevSys &d = sys[s];
    const uint64_t step = d.step + (uint64_t)adv;
    const int P = sa.P, tid = threadIdx.x, lane = lane_id(), warp = tid >> 5, nw = blockDim.x >> 5;
    int *mr = mr_out + (size_t)s * P * 3, *mnr = mnr_out + (size_t)s * P * 3;
    int *D = D_out + (size_t)s * Dcap * 3, *cr = cr_out + (size_t)s * Dcap, *cnr = cnr_out + (size_t)s * Dcap;
    int4 *pm_s = pm + (size_t)s * P;
    double *pw_s = pw + (size_t)s * P, *pg_s = pg + (size_t)s * P;
    double *pu_s = pu + (size_t)s * P, *pun_s = pun + (size_t)s * P;
    if (tid < 3) sh.L[tid] = d.L[tid];
    __syncthreads();
    if ((d.flags & FLAG_BOX) || live_n(d) == 0) {   // empty slot, or invalid box (the step is reported as failed)
        if (tid == 0) { d.nD = 0; d.nacc_r = 0; d.nacc_nr = 0; }
        return;
    }

    // 1. 1D lattice sums (k_samp_sums) and the normalizers (a tilted cell:
    // the sums over Z^3 of k_tri_reduce)
    if (warp == 0) {
        double sr = 0.0, snr = 0.0;
        if (d.tri) {
            for (int l = 0; l < sa.M; ++l) {
                sr += ss[s].tHr[l];
                snr += ss[s].tHnr[l];
            }
        } else {
            load_sums(sa, ss[s], sh.L, sh, sr, snr);
        }
        if (lane == 0) {
            sh.Sr = sr; sh.Snr = snr;
            d.Sr = sr; d.Snr = snr;
            cnt_r = 0; cnt_nr = 0;
        }
    }
    __syncthreads();

    // 2. exact draws
    if (sa.kind == 0) {
        if (tid == 0) {                       // drawn by k_samp_prop
            start_m[0] = ss[s].start_m[0]; start_m[1] = ss[s].start_m[1]; start_m[2] = ss[s].start_m[2];
            start_w = ss[s].start_w;
            start_g = ss[s].start_g;
        }
    } else {
        for (int t = warp; t < P; t += nw) {
            uint64_t wds[4];
            int m[3];
            draw4(sa.seed, d.rng_id, step, PUR_START, (uint64_t)t, wds);
            exact_draw_warp(sa, sh, wds, false, m);
            if (lane == 0) { mr[3 * t] = m[0]; mr[3 * t + 1] = m[1]; mr[3 * t + 2] = m[2]; }
            if (sa.kind == 1) {
                draw4(sa.seed, d.rng_id, step, PUR_NR_IID, (uint64_t)t, wds);
                exact_draw_warp(sa, sh, wds, true, m);
                if (lane == 0) { mnr[3 * t] = m[0]; mnr[3 * t + 1] = m[1]; mnr[3 * t + 2] = m[2]; }
            }
        }
        if (sa.kind == 2 && warp == 0) {
            uint64_t wds[4];
            int m[3];
            draw4(sa.seed, d.rng_id, step, PUR_NR_IID, 0, wds);
            exact_draw_warp(sa, sh, wds, true, m);
            if (lane == 0) {
                double pr, pnr;
                targets(sa, sh.L, m, pr, pnr);
                nrstart_m[0] = m[0]; nrstart_m[1] = m[1]; nrstart_m[2] = m[2];
                nrstart_g = pnr / pr;
            }
        }
    }
    __syncthreads();

    // 3. proposal weights (parallel) and uniforms; the paper sampler's are
    // formed by k_samp_prop
    for (int t = tid; t < P && sa.kind != 0; t += blockDim.x) {
        uint64_t wds[4];
        int m[3];
        if (sa.kind == 0) {
            draw4(sa.seed, d.rng_id, step, PUR_PROPOSAL, (uint64_t)t, wds);
            double z[3];
            {
                double u1 = u01(wds[0]), u2 = u01(wds[1]);
                double rr = sqrt(-2.0 * log(u1)), ang = kTwoPi * u2;
                z[0] = rr * cos(ang);
                z[1] = rr * sin(ang);
                u1 = u01(wds[2]); u2 = u01(wds[3]);
                rr = sqrt(-2.0 * log(u1)); ang = kTwoPi * u2;
                z[2] = rr * cos(ang);
            }
            for (int a = 0; a < 3; ++a) m[a] = (int)floor(sh.L[a] * (z[a] * sa.sig_u) + 0.5);
            double w = 0.0, g = 0.0;
            if (m[0] || m[1] || m[2]) {
                double pr, pnr;
                targets(sa, sh.L, m, pr, pnr);
                w = pr / qprop(sa, sh.L, m);
                g = pnr / pr;
            }
            pm_s[t] = make_int4(m[0], m[1], m[2], 0);
            pw_s[t] = w;
            pg_s[t] = g;
        } else if (sa.kind == 2) {
            m[0] = mr[3 * t]; m[1] = mr[3 * t + 1]; m[2] = mr[3 * t + 2];
            double pr, pnr;
            targets(sa, sh.L, m, pr, pnr);
            pg_s[t] = pnr / pr;
        }
        draw4(sa.seed, d.rng_id, step, PUR_ACCEPT, (uint64_t)t, wds);
        pu_s[t] = u01(wds[0]);
        pun_s[t] = u01(wds[1]);
    }
    __syncthreads();

    // 4. chains: the radial chain on warp 0 and the recalibration chain on
    // warp 1, one block of 32 steps behind it (its proposals are the radial
    // states), so that the two run side by side.  Within a block a lane holds
    // one step's operands and the accept tests run in order with them
    // broadcast by shuffles, so every decision sees the same operands as a
    // sequential loop.
    __shared__ int xs[2][32][3];              // radial states of a block (double buffer)
    __shared__ double xg[2][32];              // and their g = P^nr / P^r
    if (sa.kind != 1) {
        const int nb = (P + 31) / 32;
        int cur = -1, nacc = 0;               // warp 0: proposal index of the current radial state
        double wcur = start_w;
        int ym0 = 0, ym1 = 0, ym2 = 0, nn = 0;    // warp 1: current recalibration state
        double gcur = 0.0;
        if (sa.kind == 2) { ym0 = nrstart_m[0]; ym1 = nrstart_m[1]; ym2 = nrstart_m[2]; gcur = nrstart_g; }
        for (int bk = 0; bk <= nb; ++bk) {
            if (warp == 0 && bk < nb) {
                const int t0 = 32 * bk, t = t0 + lane, nt = min(32, P - t0);
                const bool valid = t < P;
                int m0, m1, m2;
                double gt;
                if (sa.kind == 0) {
                    const double u = valid ? pu_s[t] : 0.0, w = valid ? pw_s[t] : 0.0;
                    int mysrc = -1;
                    for (int j = 0; j < nt; ++j) {
                        const double uj = __shfl_sync(0xffffffffu, u, j), wj = __shfl_sync(0xffffffffu, w, j);
                        if (uj * wcur < wj) { cur = t0 + j; wcur = wj; ++nacc; }
                        if (lane == j) mysrc = cur;
                    }
                    int4 mm = make_int4(start_m[0], start_m[1], start_m[2], 0);
                    gt = start_g;
                    if (valid && mysrc >= 0) { mm = pm_s[mysrc]; gt = pg_s[mysrc]; }
                    m0 = mm.x; m1 = mm.y; m2 = mm.z;
                    if (valid) { mr[3 * t] = m0; mr[3 * t + 1] = m1; mr[3 * t + 2] = m2; }
                } else {
                    m0 = valid ? mr[3 * t] : 0; m1 = valid ? mr[3 * t + 1] : 0; m2 = valid ? mr[3 * t + 2] : 0;
                    gt = valid ? pg_s[t] : 0.0;
                }
                xs[bk & 1][lane][0] = m0; xs[bk & 1][lane][1] = m1; xs[bk & 1][lane][2] = m2;
                xg[bk & 1][lane] = gt;
            }
            if (warp == 1 && bk >= 1) {
                const int b1 = bk - 1, t0 = 32 * b1, t = t0 + lane, nt = min(32, P - t0);
                const bool valid = t < P;
                const int m0 = xs[b1 & 1][lane][0], m1 = xs[b1 & 1][lane][1], m2 = xs[b1 & 1][lane][2];
                const double gt = xg[b1 & 1][lane];
                if (b1 == 0 && sa.kind == 0) {   // y_0 = x_1: the first radial state
                    gcur = __shfl_sync(0xffffffffu, gt, 0);
                    ym0 = __shfl_sync(0xffffffffu, m0, 0);
                    ym1 = __shfl_sync(0xffffffffu, m1, 0);
                    ym2 = __shfl_sync(0xffffffffu, m2, 0);
                }
                const double un = valid ? pun_s[t] : 0.0;
                int y0 = 0, y1 = 0, y2 = 0;
                for (int j = 0; j < nt; ++j) {
                    const double uj = __shfl_sync(0xffffffffu, un, j), gj = __shfl_sync(0xffffffffu, gt, j);
                    const int c0 = __shfl_sync(0xffffffffu, m0, j), c1 = __shfl_sync(0xffffffffu, m1, j),
                              c2 = __shfl_sync(0xffffffffu, m2, j);
                    if (uj * gcur < gj) { ym0 = c0; ym1 = c1; ym2 = c2; gcur = gj; ++nn; }
                    if (lane == j) { y0 = ym0; y1 = ym1; y2 = ym2; }
                }
                if (valid) { mnr[3 * t] = y0; mnr[3 * t + 1] = y1; mnr[3 * t + 2] = y2; }
            }
            __syncthreads();
        }
        if (warp == 0 && lane == 0) cnt_r = nacc;
        if (warp == 1 && lane == 0) cnt_nr = nn;
    }
    __syncthreads();

    // 5. distinct modes: sort 2P keys (mode key << 1 | tag), bitonic in shared memory
    int n2 = 2 * P, p2 = 1;
    while (p2 < n2) p2 <<= 1;
    for (int k = tid; k < p2; k += blockDim.x) {
        uint64_t key = ~0ull;
        if (k < P) key = (mode_key(mr + 3 * k) << 1);
        else if (k < n2) key = (mode_key(mnr + 3 * (k - P)) << 1) | 1ull;
        keys[k] = key;
    }
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = tid; t < p2 / 2; t += blockDim.x) {
                int lo = 2 * j * (t / j) + (t % j), hi = lo + j;
                bool up = (lo & k) == 0;
                uint64_t x = keys[lo], y = keys[hi];
                if ((x > y) == up) { keys[lo] = y; keys[hi] = x; }
            }
            __syncthreads();
        }
    }
    // 6. segment heads, their ranks by a block scan, multiplicities by a walk
    // over each (short) segment: within a segment the radial entries (tag 0)
    // precede the recalibrated ones (tag 1)
    const int per = (n2 + blockDim.x - 1) / blockDim.x;
    const int k0 = min(n2, tid * per), k1 = min(n2, k0 + per);
    int nh = 0;
    for (int k = k0; k < k1; ++k) nh += (k == 0 || (keys[k] >> 1) != (keys[k - 1] >> 1));
    int incl = nh;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) scan_w[warp] = incl;
    __syncthreads();
    int base = incl - nh;
    for (int w = 0; w < warp; ++w) base += scan_w[w];
    for (int k = k0; k < k1; ++k) {
        const uint64_t mk = keys[k] >> 1;
        if (k > 0 && mk == (keys[k - 1] >> 1)) continue;
        int e = k, nr0 = 0, nr1 = 0;
        while (e < n2 && (keys[e] >> 1) == mk) {
            if (keys[e] & 1ull) ++nr1; else ++nr0;
            ++e;
        }
        int m[3];
        key_mode(mk, m);
        D[3 * base] = m[0]; D[3 * base + 1] = m[1]; D[3 * base + 2] = m[2];
        cr[base] = nr0; cnr[base] = nr1;
        ++base;
    }
    if (tid == blockDim.x - 1) {
        d.nD = base;                          // the last thread ends after every head
        d.nacc_r = cnt_r;
        d.nacc_nr = cnt_nr;
    }
}

// Lattice sums of a tilted cell, once per cell.  k_tri_gy: one thread per
// (l, m_0, m_1), the sums over m_2 (ascending) of k_a^2 e_l and k^4 e_l;
// k_tri_reduce: one block per tilted system, Gx = sum over m_1 (ascending),
// tS = sum over m_0, the normalizer terms H^r_l = c_l (tS_0 + tS_1 + tS_2)
// and H^nr_l = c'_l sum_{m_0, m_1} G4.
__global__ void k_tri_gy(const DevSys *__restrict__ sys, const SamplerArgs sa, const SampScratch *__restrict__ ss,
                         const int *__restrict__ tri_sys)
{
    const int s = tri_sys[blockIdx.y];
    const DevSys &d = sys[s];
    const SampScratch &sc = ss[s];
    const int mm0 = sc.tmm[0], mm1 = sc.tmm[1], mm2 = sc.tmm[2];
    const int nx = 2 * mm0 + 1, ny = 2 * mm1 + 1, nz = 2 * mm2 + 1;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)sa.M * nx * ny) return;
    const int l = (int)(idx / ((long long)nx * ny)), i = (int)((idx / ny) % nx), j = (int)(idx % ny);
    double g0 = 0.0, g1 = 0.0, g2 = 0.0, g4 = 0.0;
    for (int kz = 0; kz < nz; ++kz) {
        const int m[3] = {i - mm0, j - mm1, kz - mm2};
        double k[3];
        kvec_of(d, m, k);
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        const double e = exp(-(sa.st2q[l] * k2));
        g0 += k[0] * k[0] * e;
        g1 += k[1] * k[1] * e;
        g2 += k[2] * k[2] * e;
        g4 += (k2 * k2) * e;
    }
    double *Gy = sa.tri_tab + sc.tab0;
    double *G4 = Gy + (size_t)sa.M * 3 * nx * ny + (size_t)sa.M * 3 * nx;
    Gy[(((size_t)l * 3 + 0) * nx + i) * ny + j] = g0;
    Gy[(((size_t)l * 3 + 1) * nx + i) * ny + j] = g1;
    Gy[(((size_t)l * 3 + 2) * nx + i) * ny + j] = g2;
    G4[((size_t)l * nx + i) * ny + j] = g4;
}

__global__ void k_tri_reduce(const SamplerArgs sa, SampScratch *__restrict__ ss, const int *__restrict__ tri_sys)
{
    SampScratch &sc = ss[tri_sys[blockIdx.x]];
    const int nx = 2 * sc.tmm[0] + 1, ny = 2 * sc.tmm[1] + 1;
    const double *Gy = sa.tri_tab + sc.tab0;
    double *Gx = sa.tri_tab + sc.tab0 + (size_t)sa.M * 3 * nx * ny;
    const double *G4 = Gx + (size_t)sa.M * 3 * nx;
    for (int r = threadIdx.x; r < sa.M * 3 * nx; r += blockDim.x) {
        double a = 0.0;
        for (int j = 0; j < ny; ++j) a += Gy[(size_t)r * ny + j];
        Gx[r] = a;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < sa.M * 3; r += blockDim.x) {
        double a = 0.0;
        for (int i = 0; i < nx; ++i) a += Gx[(size_t)r * nx + i];
        sc.tS[r / 3][r % 3] = a;
    }
    for (int l = threadIdx.x; l < sa.M; l += blockDim.x) {
        double a = 0.0;
        for (size_t u = 0; u < (size_t)nx * ny; ++u) a += G4[(size_t)l * nx * ny + u];
        sc.tHnr[l] = sa.cn[l] * a;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < sa.M; l += blockDim.x) sc.tHr[l] = sa.cr[l] * (sc.tS[l][0] + sc.tS[l][1] + sc.tS[l][2]);
}

void launch_tri_tables(const Batch &b, const SamplerArgs &sa, SampScratch *ss, const int *tri_sys, int ntri,
                       const int *mm_max, cudaStream_t st)
{
    (void)b;
    if (ntri == 0) return;
    const long long n = (long long)sa.M * (2 * mm_max[0] + 1) * (2 * mm_max[1] + 1);
    k_tri_gy<<<dim3((unsigned)((n + 127) / 128), ntri), 128, 0, st>>>(b.sys, sa, ss, tri_sys);
    k_tri_reduce<<<ntri, 256, 0, st>>>(sa, ss, tri_sys);
}

static size_t sampler_smem(int P)
{
    int p2 = 1;
    while (p2 < 2 * P) p2 <<= 1;
    return (size_t)p2 * sizeof(uint64_t);
}

cudaError_t prepare_sampler(int P)
{
    return cudaFuncSetAttribute(k_sampler, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sampler_smem(P));
}

void launch_sampler(const Batch &b, const SamplerArgs &sa, int adv, int *mr, int *mnr, int *D, int *cr,
                    int *cnr, int4 *pm, double *pw, double *pg, double *pu, double *pun, SampScratch *ss,
                    int Dcap, cudaStream_t st)
{
    k_samp_sums<<<dim3(b.S, 3 * sa.M), 32, 0, st>>>(b.sys, sa, ss);
    if (sa.kind == 0) {
        k_samp_prop<<<dim3(b.S, sa.P + 1), 32, 0, st>>>(b.sys, sa, adv, ss, pm, pw, pg, pu, pun);
        if (sa.has_tri)
            k_samp_prop_tri<<<dim3(b.S, sa.P + 1), 32, 0, st>>>(b.sys, sa, adv, ss, pm, pw, pg, pu, pun);
    }
    k_sampler<<<b.S, 256, sampler_smem(sa.P), st>>>(b.sys, sa, adv, mr, mnr, D, cr, cnr, pm, pw, pg, pu, pun, ss,
                                                    Dcap);
}

}  // namespace rbsog
