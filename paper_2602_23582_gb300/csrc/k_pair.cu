// k_pair.cu -- SOG short-range pair forces, energy and virial over cell lists
// (paper sec. 2.2 and 3.1; eqs. force_SOG, U_short, P_short) plus a 12-6
// Lennard-Jones term cut (unshifted) at r_c.
//
// Per pair with r < r_c and different molecule ids:
//   f   = ke q_i q_j (1/r^3 - sum_{l<M} w~_l e^{-r^2/s~_l^2}) r_vec   (kernel N~)
//   U  += ke q_i q_j (1/r   - sum_{l<ME} w_l e^{-r^2/s_l^2})          (kernel N)
//   W  += f (x) r_vec  (eq. P_short: P^N = W / V)
//
// Both builds evaluate every pair once (Newton's third law) and add forces
// as 64-bit fixed point, so sums do not depend on the order of the adds.
// FP32 build: one fused kernel over clusters of 4 atoms (k_pair_cluster).
// FP64 build: one warp per (32-atom group, dz plane, cell quarter), hits
// queued per lane and evaluated with full lanes (k_pair_f64).
//
// Coordinates are cell-local.  A neighbour cell's periodic offset d_a w_a is
// split into FP32 hi + lo parts: the evaluation subtracts both, so that the
// rounding of w_a does not shift every cross-cell distance the same way (a
// systematic error that the r^-12 and 1/r - F(r) terms would amplify).
#include "internal.h"

namespace rbsog {

namespace {

constexpr int QCAP = 64;      // FP64 kernel: the warp's hit queue (power of two; < 32 pending before a push of <= 32)
constexpr int kMaxPlane = 32; // neighbour cells of one dz plane (25 for cells of r_c/2)
constexpr int kMaxNb = 128;   // neighbour cells of the stencil (125 for cells of r_c/2)

size_t pair_smem(int precision)
{
    return (size_t)kPairWarps * (QCAP * sizeof(uint2) + kMaxPlane * 16);
}

__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

struct AccD {
    double uc, ul;
    double w[6], wc[6], wl[6];
};

// Cutoff decision for a pair close to r_c, in FP64 from the original
// positions with the minimum image, as the CPU reference decides it.
// (out of line: the call sits in a branch taken a few times per launch, and an
// inlined body costs the common path registers and instructions)
__device__ __noinline__ bool inside_cutoff_fp64(const double *__restrict__ r, int i, int j, const DevSys &d,
                                                double rc2)
{
    double r2 = 0.0;
    if (d.tri) {
        double dd[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
        min_image_tri(d, dd);
        r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
    } else {
        for (int a = 0; a < 3; ++a) {
            double dd = r[3 * i + a] - r[3 * j + a];
            dd = d.L[a] * (dd / d.L[a] - rint(dd / d.L[a]));
            r2 += dd * dd;
        }
    }
    return r2 < rc2;
}

// 2^x for x <= 0 without the MUFU approximation: x = n + f, n = rint(x),
// |f| <= 1/2, 2^f from its Taylor series sum_k (f ln 2)^k / k! to degree 9
// (remainder < 0.35^10 / 10! ~ 8e-12), Horner with FMA (rounding errors of
// either sign), 2^n by an exponent add.  Used where a bias shared by all
// pairs would accumulate (the energy path).
__device__ __forceinline__ float exp2_poly(float x)
{
    x = fmaxf(x, -125.f);
    const float n = rintf(x);
    const float f = x - n;
    float p = 1.0178086e-07f;                 // (ln 2)^9 / 9!
    p = fmaf(p, f, 1.3215487e-06f);           // (ln 2)^8 / 8!
    p = fmaf(p, f, 1.5252734e-05f);           // (ln 2)^7 / 7!
    p = fmaf(p, f, 1.5403530e-04f);           // (ln 2)^6 / 6!
    p = fmaf(p, f, 1.3333558e-03f);           // (ln 2)^5 / 5!
    p = fmaf(p, f, 9.6181291e-03f);           // (ln 2)^4 / 4!
    p = fmaf(p, f, 5.5504109e-02f);           // (ln 2)^3 / 3!
    p = fmaf(p, f, 2.4022651e-01f);           // (ln 2)^2 / 2!
    p = fmaf(p, f, 6.9314718e-01f);           // ln 2
    p = fmaf(p, f, 1.0f);
    return __int_as_float(__float_as_int(p) + ((int)n << 23));
}

// One FP64 pair (i, j) with d = r_i - r_j: returns f (force on i = f d)
// and adds energies and virials (EN: also the Coulomb / LJ split and the
// energies; the total virial W always).
template <bool EN>
__device__ __forceinline__ double pair_eval_d(const PairConstsD &pc, double dx, double dy, double dz, double r2,
                                              double qq, double2 lab, AccD &acc)
{
    const double rinv = rsqrt(r2);
    const double r2inv = rinv * rinv;
    double st = pc.tt[kTailD], se = pc.te[kTailD];
#pragma unroll
    for (int k = kTailD - 1; k >= 0; --k) {
        st = fma(st, r2, pc.tt[k]);
        if (EN) se = fma(se, r2, pc.te[k]);
    }
    for (int l = 0; l < pc.nf; ++l) {
        const double e = exp(-r2 * pc.inv_s2[l]);
        st = fma(pc.wt[l], e, st);
        if (EN) se = fma(pc.w[l], e, se);
    }
    const double fc = qq * (r2inv * rinv - st);
    const double r6inv = r2inv * r2inv * r2inv;
    const double fl = (12.0 * lab.x * r6inv - 6.0 * lab.y) * r6inv * r2inv;
    const double f = fc + fl;
    acc.w[0] = fma(f * dx, dx, acc.w[0]); acc.w[1] = fma(f * dy, dy, acc.w[1]); acc.w[2] = fma(f * dz, dz, acc.w[2]);
    acc.w[3] = fma(f * dx, dy, acc.w[3]); acc.w[4] = fma(f * dx, dz, acc.w[4]); acc.w[5] = fma(f * dy, dz, acc.w[5]);
    if (EN) {
        acc.uc += qq * (rinv - se);
        acc.ul += (lab.x * r6inv - lab.y) * r6inv;
        acc.wc[0] += fc * dx * dx; acc.wc[1] += fc * dy * dy; acc.wc[2] += fc * dz * dz;
        acc.wc[3] += fc * dx * dy; acc.wc[4] += fc * dx * dz; acc.wc[5] += fc * dy * dz;
        acc.wl[0] += fl * dx * dx; acc.wl[1] += fl * dy * dy; acc.wl[2] += fl * dz * dz;
        acc.wl[3] += fl * dx * dy; acc.wl[4] += fl * dx * dz; acc.wl[5] += fl * dy * dz;
    }
    return f;
}

__device__ __forceinline__ int wrapi(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// f added to a force of the FP64 build: two 64-bit fixed-point words, the
// value in units of 2^-40 rounded to an integer and the rest in units of
// 2^-80 (integer sums are exact and order-independent).
// The words are formed from the bits of f with integer instructions only
// (the FP64 pipe, which bounds this kernel, is left to the arithmetic):
// |f| = m 2^(e - 52), so |f| 2^80 = m 2^(e + 28) as a 128-bit integer U
// (rounded to an integer, ties away from zero, when e + 28 < 0); the words
// are U >> 40 and U mod 2^40, negated as one 128-bit number for f < 0 (the
// second word then stays in [0, 2^40)).  |f| >= 2^23 saturates.
__device__ __forceinline__ void add_fix2(unsigned long long *hi, unsigned long long *lo, double f)
{
    const long long b = __double_as_longlong(f);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    const unsigned long long m = ((unsigned long long)b & 0xfffffffffffffull) | 0x10000000000000ull;
    const int sh = e + 28;
    unsigned long long uh, ul;                         // U = uh 2^64 + ul
    if (sh >= 0) {
        if (sh < 51) {
            uh = sh == 0 ? 0ull : m >> (64 - sh);
            ul = m << sh;
        } else {
            uh = 0x7fffffull;                          // saturate: 2^(63 + 40 - 64) - 1
            ul = ~0ull;
        }
    } else {
        uh = 0ull;
        ul = sh > -54 ? (m + (1ull << (-sh - 1))) >> -sh : 0ull;
    }
    const unsigned long long mask = (1ull << 40) - 1ull;
    long long h = (long long)((uh << 24) | (ul >> 40));
    long long l = (long long)(ul & mask);
    if (b < 0) {                                       // -U: borrow from the high word when l != 0
        h = l ? -h - 1 : -h;
        l = l ? (long long)(mask + 1ull) - l : 0;
    }
    atomicAdd(hi, (unsigned long long)h);
    atomicAdd(lo, (unsigned long long)l);
}

}  // namespace

// ---------------------------------------------------------------------------
// FP32 path: one fused kernel over clusters, each pair evaluated once.
//
// Work unit = one warp = i-cluster I (kClus = 4 consecutive cell-sorted atoms
// of one cell) x dz plane p = 0..sub of the half stencil: the neighbour cells
// (dx, dy, p) with p > 0, or p = 0 and (dy > 0 or dy = 0 and dx > 0), and on
// plane 0 the clusters J > I of I's own cell plus the pairs inside I.  Every
// unordered pair of atoms within r_c is seen exactly once.
//
// The clusters of the unit's cells are numbered consecutively; the warp
// tests them 32 at a time against I by their bounding boxes (each lane finds
// its candidate's cell by bisection over the cells' first numbers, held one
// per lane; the passing clusters are appended to a small queue in shared
// memory) and evaluates them in rounds of 8 tiles: lane
// (g, k) of the 8 four-lane groups holds atom k of I and, in step t = 0..3,
// pairs it with atom (k + t) mod 4 of the group's cluster J, so each group
// evaluates its 4 x 4 tile with full lanes.  The force on I accumulates in
// registers over the whole unit; the force on J's atoms travels with them
// (after each step the running sum moves one lane down, to the lane that meets
// that atom next), so after the fourth step each lane holds one J atom's total
// over the tile and adds it to the force buffer.  Forces are accumulated as
// 64-bit fixed point (units of 2^-32 kcal/mol/A): integer additions are
// exact and commute, so the sum does not depend on the order in which the
// warps reach an atom, and results are deterministic.  Energies (and, with
// energies, the virial and its Coulomb / LJ split) are summed per lane in the
// warp's fixed pair order and reduced to one record per warp.  Force-only
// evaluations form the virial sum_pairs r_ij (x) f_ij from the force sums the
// kernel holds anyway: sum_i x_i (x) F_i over the unit (I's cell frame) plus,
// per tile, sum_j (x_j + o) (x) F_j with o J's cell offset (the same sum by
// F_i = sum_j f_ij, F_j = -sum_i f_ij; 9 operations per lane and tile instead
// of 9 per pair).
// ---------------------------------------------------------------------------
namespace {

constexpr int kQueue = 64;           // tile queue per warp (entries in flight <= 7 + 32)

struct TileAcc {
    float fx, fy, fz;                // force on this lane's i atom
    float w[6];                      // total virial
    float uc, ul, uq, cuc, cul, cuq; // energies, sum q_i q_j (EN), with compensation terms
    float wc[6], wl[6];              // Coulomb / LJ split of the virial (EN)
};

// f 2^32 as a 64-bit integer in two 32-bit conversions: the high word
// floor(f), the low word (f - floor(f)) 2^32 rounded (f - floor(f) rounds up
// to 1 only for f just below an integer, and the low word then saturates at
// 2^32 - 1: one unit off).  The float-to-int64 conversion it replaces issues to
// this part's FP64 pipe, whose latency the atomic add then waits for: water
// pair launch 97.4 -> 95.0 us.  Any fixed rounding keeps the sums exact and
// order-independent; the words resolve 2^-24 of a unit force for -1 < f < 0.
__device__ __forceinline__ long long to_fix(float f)
{
    const float h = floorf(f);
    const int hi = __float2int_rn(h);
    const unsigned lo = __float2uint_rn((f - h) * (float)kFixScale);
    return (long long)(((unsigned long long)(unsigned)hi << 32) | lo);
}

// One 4 x 4 tile: this lane's atom i (cell-local xi, already shifted by the
// high part of J's cell offset) against atom (k + t) mod 4 of J in step t.
// DIAG: J = I (steps 1..3 only; every unordered pair is met twice, from each
// side, so it adds to the force on i only and counts half in energy and
// virial).  Returns with fj = the force on J atom (k + 3) mod 4 over the tile.
template <int NF, bool EN, bool DIAG>
__device__ __forceinline__ void tile(const PairConstsF &pc, float xs, float ys, float zs, float4 ol, int moli,
                                     float qi, int ai, int jslot, int jfirst, int kk, int gbase,
                                     const float4 *__restrict__ pos4, const float2 *__restrict__ qt,
                                     const float2 *__restrict__ ljrow, const float2 *__restrict__ ljlorow,
                                     const int *__restrict__ sidx, const double *__restrict__ r, const DevSys &dsys,
                                     TileAcc &acc, float &fjx, float &fjy, float &fjz, float4 &pjl)
{
    fjx = fjy = fjz = 0.f;
#pragma unroll
    for (int t = DIAG ? 1 : 0; t < 4; ++t) {
        // atom (k + t) mod 4 of J; slots past a cluster's atoms hold a far-away
        // atom of no molecule, which no cutoff test passes
        const int jj = (kk + t) & 3;
        const float4 pj = pos4[jslot + jj];
        if (t == 3) pjl = pj;                          // the atom whose sum this lane ends with
        const float2 qj = qt[jslot + jj];
        const int aj = jfirst + jj;
        const float dx = (xs - pj.x) - ol.x, dy = (ys - pj.y) - ol.y, dz = (zs - pj.z) - ol.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        // with energies, pairs within a relative 1e-5 of r_c^2 are decided in
        // FP64 from the original positions (the energy kernel N is about 2e-3 / A
        // at r_c, so one pair on the wrong side shifts U by ~ke q_i q_j 2e-3);
        // force-only evaluations decide in FP32: the force kernel N~ is ~5e-9 at
        // r_c, and a pair within FP32 rounding of r_c moves a force by at most
        // the LJ force there
        bool in;
        if (EN) {
            in = r2 < pc.rc2_lo;
            const bool near = !in && r2 < pc.rc2_hi;
            if (__any_sync(0xffffffffu, near)) {         // rare: out of the common path
                if (near) in = inside_cutoff_fp64(r, sidx[ai], sidx[aj], dsys, pc.rc2d);
            }
        } else {
            in = r2 < pc.rc2;
        }
        in = in && __float_as_int(pj.w) != moli;       // pairs of one molecule are excluded
        // (a pair that is not inside may give non-finite values here, e.g. two
        // padding atoms at one place: its force is selected away below)
        float rinv = rsqrt_approx(r2);
        rinv = rinv * fmaf(-0.5f * r2 * rinv, rinv, 1.5f);
        const float r2inv = rinv * rinv;
        float st = pc.tt[kTailF];
#pragma unroll
        for (int k = kTailF - 1; k >= 0; --k) st = fmaf(st, r2, pc.tt[k]);
        if (NF > 0) {
#pragma unroll
            for (int l = 0; l < NF; ++l) st = fmaf(pc.wt[l], ex2f(-r2 * pc.beta[l]), st);
        } else {
            for (int l = 0; l < pc.nff; ++l) st = fmaf(pc.wt[l], ex2f(-r2 * pc.beta[l]), st);
        }
        const float qq = qi * qj.x;                    // qi holds ke q_i
        const float fc = qq * (r2inv * rinv - st);
        const int tj = __float_as_int(qj.y);
        const float2 lab = ljrow[tj];   // EN: (4 eps s^12, 4 eps s^6); else (48 eps s^12, 24 eps s^6)
        const float r6inv = r2inv * r2inv * r2inv;
        const float fl = EN ? (12.f * lab.x * r6inv - 6.f * lab.y) * r6inv * r2inv
                            : fmaf(lab.x, r6inv, -lab.y) * r6inv * r2inv;
        const float f = in ? fc + fl : 0.f;
        acc.fx = fmaf(f, dx, acc.fx);
        acc.fy = fmaf(f, dy, acc.fy);
        acc.fz = fmaf(f, dz, acc.fz);
        if (EN) {                                      // per-pair virial (force-only: from the sums, below)
            const float fw = DIAG ? 0.5f * f : f;
            const float gx = fw * dx, gy = fw * dy;
            acc.w[0] = fmaf(gx, dx, acc.w[0]); acc.w[1] = fmaf(gy, dy, acc.w[1]);
            acc.w[2] = fmaf(fw * dz, dz, acc.w[2]); acc.w[3] = fmaf(gx, dy, acc.w[3]);
            acc.w[4] = fmaf(gx, dz, acc.w[4]); acc.w[5] = fmaf(gy, dz, acc.w[5]);
        }
        if (EN && in) {
            // energy kernel N(r) = 1/r - F(r); the constant of the tail is
            // applied to sum q_i q_j in FP64 by the caller
            const float h = DIAG ? 0.5f : 1.f;
            float se = pc.te[kTail];
#pragma unroll
            for (int k = kTail - 1; k >= 1; --k) se = fmaf(se, r2, pc.te[k]);
            se *= r2;
            for (int l = 0; l < pc.nfe; ++l) {
                const float e = exp2_poly(fmaf(-r2, pc.be_hi[l], -r2 * pc.be_lo[l]));
                se = fmaf(pc.w_hi[l], e, fmaf(pc.w_lo[l], e, se));
            }
            kahan_add(acc.uc, acc.cuc, h * (qq * (rinv - se)));
            kahan_add(acc.uq, acc.cuq, h * qq);
            const float2 lo = ljlorow[tj];
            kahan_add(acc.ul, acc.cul, h * ((fmaf(lab.x, r6inv, -lab.y) + fmaf(lo.x, r6inv, -lo.y)) * r6inv));
            const float fcw = h * fc, flw = h * fl;
            const float cx = fcw * dx, cy = fcw * dy, lx = flw * dx, ly = flw * dy;
            acc.wc[0] = fmaf(cx, dx, acc.wc[0]); acc.wc[1] = fmaf(cy, dy, acc.wc[1]);
            acc.wc[2] = fmaf(fcw * dz, dz, acc.wc[2]); acc.wc[3] = fmaf(cx, dy, acc.wc[3]);
            acc.wc[4] = fmaf(cx, dz, acc.wc[4]); acc.wc[5] = fmaf(cy, dz, acc.wc[5]);
            acc.wl[0] = fmaf(lx, dx, acc.wl[0]); acc.wl[1] = fmaf(ly, dy, acc.wl[1]);
            acc.wl[2] = fmaf(flw * dz, dz, acc.wl[2]); acc.wl[3] = fmaf(lx, dy, acc.wl[3]);
            acc.wl[4] = fmaf(lx, dz, acc.wl[4]); acc.wl[5] = fmaf(ly, dz, acc.wl[5]);
        }
        if (!DIAG) {
            fjx = fmaf(-f, dx, fjx);
            fjy = fmaf(-f, dy, fjy);
            fjz = fmaf(-f, dz, fjz);
            if (t < 3) {                               // hand the sums to the lane that meets these atoms next
                const int src = gbase + ((kk + 1) & 3);
                fjx = __shfl_sync(0xffffffffu, fjx, src);
                fjy = __shfl_sync(0xffffffffu, fjy, src);
                fjz = __shfl_sync(0xffffffffu, fjz, src);
            }
        }
    }
}

}  // namespace

template <int NF, bool EN>
__global__ void __launch_bounds__(32 * kCpWarps, EN ? 5 : 8)
k_pair_cluster(const DevSys *__restrict__ sys, const int *__restrict__ item_sys, const int2 *__restrict__ items,
               const int2 *__restrict__ ccl, const float4 *__restrict__ cbox, const float4 *__restrict__ pos4,
               const float2 *__restrict__ qt, const float2 *__restrict__ lj, const float2 *__restrict__ ljlo,
               const int *__restrict__ sidx, const double *__restrict__ r, int sub, int N, int item_cap,
               unsigned long long *__restrict__ ffix, double *__restrict__ partial, const PairConstsF pc)
{
    __shared__ float4 offh[kMaxNb], offl[kMaxNb];
    __shared__ float2 ljs[EN ? 2 : 1][kMaxTypes * kMaxTypes];   // the system's LJ table (and remainders)
    __shared__ int2 queue[kCpWarps][kQueue];
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const int kk = lane & 3, gbase = lane & ~3, grp = lane >> 2;
    const int span = 2 * sub + 1, nparts = pair_parts(1, sub);
    // units: item-major, kCpWarps per block; a system's item range is a
    // multiple of kCpWarps items, so a block never mixes systems
    const int unit = blockIdx.x * kCpWarps + warp;
    const int it = unit / nparts, part = unit % nparts;
    const DevSys &d = sys[item_sys[(blockIdx.x * kCpWarps) / nparts]];
    const bool ok = !(d.flags & FLAG_OVERFLOW) && live_n(d) > 0;   // block-uniform
    if (ok) {
        // neighbour-cell offsets d_a w_a as FP32 hi + lo (the rounding of w
        // must not shift every cross-cell distance the same way)
        for (int nb = threadIdx.x; nb < span * span * span; nb += blockDim.x) {
            // h (delta / n): the diagonal part and the tilt terms (zero when orthorhombic)
            const int ex = nb % span - sub, ey = (nb / span) % span - sub, ez = nb / (span * span) - sub;
            const double ox = ex * d.w[0] + (ey * d.tw[0] + ez * d.tw[1]), oy = ey * d.w[1] + ez * d.tw[2],
                         oz = ez * d.w[2];
            const float hx = (float)ox, hy = (float)oy, hz = (float)oz;
            offh[nb] = make_float4(hx, hy, hz, 0.f);
            offl[nb] = make_float4((float)(ox - (double)hx), (float)(oy - (double)hy), (float)(oz - (double)hz), 0.f);
        }
        for (int t = threadIdx.x; t < d.ntypes * d.ntypes; t += blockDim.x) {
            const float2 v = lj[d.lj0 + t];
            ljs[0][t] = EN ? v : make_float2(12.f * v.x, 6.f * v.y);
            if (EN) ljs[EN ? 1 : 0][t] = ljlo[d.lj0 + t];
        }
    }
    __syncthreads();
    TileAcc acc;
    acc.fx = acc.fy = acc.fz = 0.f;
    acc.uc = acc.ul = acc.uq = acc.cuc = acc.cul = acc.cuq = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) acc.w[k] = acc.wc[k] = acc.wl[k] = 0.f;
    const int2 item = items[it];
    if (ok && item.x >= 0 && it - d.item0 < d.nitems) {     // warp-uniform
        const int gc = item.x;
        const int n0 = d.ncell[0], n1 = d.ncell[1], n2 = d.ncell[2];
        const int lc = gc - d.cell0;
        const int cx = lc % n0, cy = (lc / n0) % n1, cz = lc / (n0 * n1);
        const float4 bi0 = cbox[2 * it], bi1 = cbox[2 * it + 1];
        const int ifirst = __float_as_int(bi0.w), ni = __float_as_int(bi1.w);
        const bool vi = kk < ni;
        const int ai = ifirst + (vi ? kk : 0);
        const float4 pi = pos4[kClus * it + kk];
        const float2 qi2 = qt[kClus * it + kk];
        const int moli = __float_as_int(pi.w);
        const float qi = pc.ke * qi2.x;
        const int rowi = __float_as_int(qi2.y) * d.ntypes;
        const float2 *ljrow = ljs[0] + rowi, *ljlorow = ljs[EN ? 1 : 0] + rowi;
        unsigned long long *const fxs = ffix, *const fys = ffix + N, *const fzs = ffix + 2 * (size_t)N;
        float fjx, fjy, fjz;
        float4 pjl;
        // the pairs inside I (plane 0), by the first group; the whole warp
        // runs the tile (its votes need every lane), the other groups against
        // the dummy cluster, which adds nothing
        if (part == 0)
            tile<NF, EN, true>(pc, pi.x, pi.y, pi.z, make_float4(0.f, 0.f, 0.f, 0.f), moli, qi, ai,
                               kClus * (grp == 0 ? it : item_cap), ifirst, kk, gbase, pos4, qt, ljrow, ljlorow,
                               sidx, r, d, acc, fjx, fjy, fjz, pjl);
        // candidate cells, one per lane: plane 0 (I's own cell -- its clusters
        // after I -- then the upper half), then with one unit per cluster
        // (cells of r_c) the planes above
        const int nc0 = sub * (span + 1) + 1;
        const int ncand = nparts == 1 ? nc0 + span * span : (part == 0 ? nc0 : span * span);
        int cj = 0, cn = 0, cnb = 0;
        if (lane < ncand) {
            int ddx, ddy, pz;
            const int c0 = nparts == 1 ? lane : (part == 0 ? lane : nc0 + lane);
            if (c0 < nc0) {
                pz = 0;
                if (c0 == 0) { ddx = 0; ddy = 0; }
                else if (c0 <= sub) { ddx = c0; ddy = 0; }
                else { const int u = c0 - sub - 1; ddx = u % span - sub; ddy = u / span + 1; }
            } else {
                const int u = c0 - nc0;
                pz = nparts == 1 ? 1 + u / (span * span) : part;
                const int v = u % (span * span);
                ddx = v % span - sub; ddy = v / span - sub;
            }
            const int g = d.cell0 + wrapi(cx + ddx, n0) + n0 * (wrapi(cy + ddy, n1) + n1 * wrapi(cz + pz, n2));
            const int2 cc = ccl[g];
            cj = cc.x;
            cn = cc.y;
            if (c0 == 0) { cj = it + 1; cn = cc.x + cc.y - (it + 1); }
            cnb = (pz + sub) * span * span + (ddy + sub) * span + (ddx + sub);
        }
        int incl = cn;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int cbase = lane < ncand ? incl - cn : 0x7fffffff;   // first candidate of this lane's cell
        // box test at r_c (tiles are formed anew every evaluation), with a
        // margin far above the rounding of centres and extents
        const float rl = sqrtf(pc.rc2_hi) + 1e-3f;
        const float rl2 = rl * rl;
        int2 *q = queue[warp];
        int qhead = 0, qtail = 0, k0 = 0;
        for (;;) {
            if (qtail - qhead >= 8 || (k0 >= total && qtail > qhead)) {
                // a round: group g takes queue entry qhead + g (a group
                // without one takes the dummy cluster past the last item,
                // whose slots hold far-away atoms of no molecule)
                const int qe = qhead + grp;
                int2 e = make_int2(item_cap, 0);
                if (qe < qtail) e = q[qe & (kQueue - 1)];
                qhead = min(qhead + 8, qtail);
                const int jc = e.x, code = e.y & 0x7f, nj = (unsigned)e.y >> 7;
                const float4 oh = offh[code], ol = offl[code];
                const int jfirst = nj ? __float_as_int(cbox[2 * jc].w) : 0;
                tile<NF, EN, false>(pc, pi.x - oh.x, pi.y - oh.y, pi.z - oh.z, ol, moli, qi, ai, kClus * jc,
                                    jfirst, kk, gbase, pos4, qt, ljrow, ljlorow, sidx, r, d, acc, fjx, fjy, fjz,
                                    pjl);
                if (!EN) {
                    // force-only virial, J side: (x_j + o) (x) F_j over the tile, x_j + o the
                    // image of J's atom in I's cell frame (high part of the offset)
                    const float px = pjl.x + oh.x, py = pjl.y + oh.y, pz = pjl.z + oh.z;
                    acc.w[0] = fmaf(px, fjx, acc.w[0]); acc.w[1] = fmaf(py, fjy, acc.w[1]);
                    acc.w[2] = fmaf(pz, fjz, acc.w[2]); acc.w[3] = fmaf(px, fjy, acc.w[3]);
                    acc.w[4] = fmaf(px, fjz, acc.w[4]); acc.w[5] = fmaf(py, fjz, acc.w[5]);
                }
                const int jl = (kk + 3) & 3;            // the J atom whose sum this lane holds
                if (jl < nj) {
                    const int aj = jfirst + jl;
                    atomicAdd(fxs + aj, (unsigned long long)to_fix(fjx));
                    atomicAdd(fys + aj, (unsigned long long)to_fix(fjy));
                    atomicAdd(fzs + aj, (unsigned long long)to_fix(fjz));
                }
                __syncwarp();
                continue;
            }
            if (k0 >= total) break;
            // a batch of 32 candidates, one per lane: find the lane's cell (the
            // last cell whose first candidate is not past it), then the
            // box-to-box distance
            const int k = k0 + lane;
            int c = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int b = __shfl_sync(0xffffffffu, cbase, c + st);
                if (b <= k) c += st;
            }
            const int jc = __shfl_sync(0xffffffffu, cj, c) + (k - __shfl_sync(0xffffffffu, cbase, c));
            const int nb = __shfl_sync(0xffffffffu, cnb, c);
            bool pass = false;
            int2 ent = make_int2(0, 0);
            if (k < total) {
                const float4 b0 = cbox[2 * jc], b1 = cbox[2 * jc + 1];
                const float4 oh = offh[nb];
                const float gx = fmaxf(fabsf((bi0.x - oh.x) - b0.x) - (bi1.x + b1.x), 0.f);
                const float gy = fmaxf(fabsf((bi0.y - oh.y) - b0.y) - (bi1.y + b1.y), 0.f);
                const float gz = fmaxf(fabsf((bi0.z - oh.z) - b0.z) - (bi1.z + b1.z), 0.f);
                pass = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < rl2;
                ent = make_int2(jc, nb | (__float_as_int(b1.w) << 7));
            }
            const unsigned m = __ballot_sync(0xffffffffu, pass);
            if (pass) q[(qtail + __popc(m & ((1u << lane) - 1u))) & (kQueue - 1)] = ent;
            qtail += __popc(m);
            k0 += 32;
            __syncwarp();
        }
        if (!EN) {
            // force-only virial, I side: x_i (x) F_i, F_i this lane's share of the force on
            // atom i over the unit (padding slots: F_i = 0 at a finite far-away x_i)
            acc.w[0] = fmaf(pi.x, acc.fx, acc.w[0]); acc.w[1] = fmaf(pi.y, acc.fy, acc.w[1]);
            acc.w[2] = fmaf(pi.z, acc.fz, acc.w[2]); acc.w[3] = fmaf(pi.x, acc.fy, acc.w[3]);
            acc.w[4] = fmaf(pi.x, acc.fz, acc.w[4]); acc.w[5] = fmaf(pi.y, acc.fz, acc.w[5]);
        }
        // the force on I's atoms: sum over the 8 groups, one add per atom
        float fx = acc.fx, fy = acc.fy, fz = acc.fz;
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
        }
        if (lane < 4 && vi) {
            atomicAdd(fxs + ai, (unsigned long long)to_fix(fx));
            atomicAdd(fys + ai, (unsigned long long)to_fix(fy));
            atomicAdd(fzs + ai, (unsigned long long)to_fix(fz));
        }
    }
    // the warp's record: virials as FP32 warp sums, energies in FP64
    // (compensated lanes) with the constant of the energy tail applied to
    // sum q_i q_j here
    double v = 0.0;
    {
        float wv[18];
#pragma unroll
        for (int k = 0; k < 6; ++k) wv[12 + k] = warp_sumf(acc.w[k]);
        double u0 = 0.0, u1 = 0.0;
        if (EN) {
            u0 = warp_sum((double)acc.uc - (double)acc.cuc - pc.te0 * ((double)acc.uq - (double)acc.cuq));
            u1 = warp_sum((double)acc.ul - (double)acc.cul);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                wv[k] = warp_sumf(acc.wc[k]);
                wv[6 + k] = warp_sumf(acc.wl[k]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) wv[k] = 0.f;
        }
        float fv = 0.f;                                // this lane's value: one conversion per lane
#pragma unroll
        for (int k = 0; k < 18; ++k)
            if (lane == 2 + k) fv = wv[k];
        v = lane == 0 ? u0 : (lane == 1 ? u1 : (double)fv);
    }
    if (lane < kPairRec) partial[(size_t)unit * kPairRec + lane] = v;
}

// ---------------------------------------------------------------------------
// FP64 kernel: one warp per (32-atom group of a cell, dz plane 0..sub of the
// half stencil, quarter of the plane's cells); every pair evaluated once.
// Lane = atom i of the group for the candidate test: the candidate atoms of
// the plane's cells are read with warp-broadcast loads and tested in FP32
// (cell-local coordinates, r^2 < 1.00001 r_c^2, different molecules); the hits
// (i, j) of all lanes go to one queue of the warp in lane order, and every 32
// of them are evaluated in FP64 with one pair per lane (the FP64 pipe of this
// part takes a warp instruction's time whatever the number of active lanes),
// with the exact cutoff test r^2 < r_c^2 in FP64.  On plane 0 the home cell
// contributes its atoms after i (cell-sorted order), and of the other cells
// those with dy > 0, or dy = 0 and dx > 0.  The forces on i and j are added
// per pair as two-word fixed point (exact, so the order of the adds does not
// matter).
// ---------------------------------------------------------------------------
template <bool EN>
__global__ void __launch_bounds__(32 * kPairWarps)
k_pair_f64(const DevSys *__restrict__ sys, const int *__restrict__ cell_sys, const int *__restrict__ start,
           const int *__restrict__ count, const int2 *__restrict__ items, const double4 *__restrict__ posd,
           const float4 *__restrict__ posf, const int2 *__restrict__ aux, const double2 *__restrict__ lj, int sub,
           int N, unsigned long long *__restrict__ ffix, double *__restrict__ partial, const PairConstsD pc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    uint2 *q = reinterpret_cast<uint2 *>(smem) + warp * QCAP;
    double2 *offp = reinterpret_cast<double2 *>(smem + kPairWarps * QCAP * sizeof(uint2)) + warp * kMaxPlane;
    const int span = 2 * sub + 1, nparts = sub + 1;
    // unit = (work item, dz plane, quarter): the quarter takes every kF64Split-th
    // cell of the plane, so that small systems still fill the SMs' FP64 pipes
    const int unit = blockIdx.x * kPairWarps + warp;
    const int2 item = items[unit / (nparts * kF64Split)];
    const int part = (unit / kF64Split) % nparts, quarter = unit % kF64Split;
    AccD acc;
    acc.uc = acc.ul = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) acc.w[k] = acc.wc[k] = acc.wl[k] = 0.0;
    // (a system with a cell beyond kCellCap atoms has failed its step: skipped)
    if (item.x >= 0 && !(sys[cell_sys[item.x]].flags & FLAG_OVERFLOW)) {
        const int gc = item.x;
        const DevSys &d = sys[cell_sys[gc]];
        const int n0 = d.ncell[0], n1 = d.ncell[1], n2 = d.ncell[2];
        const int lc = gc - d.cell0;
        const int cx = lc % n0, cy = (lc / n0) % n1, cz = lc / (n0 * n1);
        const double oz = part * d.w[2];
        const int ncand = part == 0 ? sub * (span + 1) + 1 : span * span;
        // the plane's candidate cells: (dx, dy) and their offsets
        for (int c = lane; c < ncand; c += 32) {
            int ddx, ddy;
            if (part == 0) {
                if (c == 0) { ddx = 0; ddy = 0; }
                else if (c <= sub) { ddx = c; ddy = 0; }
                else { const int u = c - sub - 1; ddx = u % span - sub; ddy = u / span + 1; }
            } else {
                ddx = c % span - sub; ddy = c / span - sub;
            }
            offp[c] = make_double2(ddx * d.w[0] + (ddy * d.tw[0] + part * d.tw[1]), ddy * d.w[1] + part * d.tw[2]);
        }
        __syncwarp();
        const int i0 = start[gc] + 32 * item.y;
        const int ni = min(32, count[gc] - 32 * item.y);
        const bool vi = lane < ni;
        float4 pif = make_float4(1e15f, 1e15f, 1e15f, 0.f);
        int moli = -0x7fffffff;
        if (vi) {
            pif = posf[i0 + lane];
            moli = aux[i0 + lane].x;
        }
        const float rc2f = pc.rc2f;
        unsigned long long *const hx = ffix, *const hy = ffix + N, *const hz = ffix + 2 * (size_t)N;
        unsigned long long *const lx = ffix + 3 * (size_t)N, *const ly = ffix + 4 * (size_t)N,
                           *const lz = ffix + 5 * (size_t)N;
        // one queue of the warp's hits (entry: j | cell code << 25, i's lane),
        // filled in lane order; every 32 entries are evaluated with one pair
        // per lane, so the FP64 instructions run with full lanes
        int head = 0, tail = 0;
        auto eval_round = [&](int n) {
            if (lane < n) {
                const uint2 e = q[(head + lane) & (QCAP - 1)];
                const int j = (int)(e.x & 0x1ffffffu), ii = i0 + (int)e.y;
                const double2 o = offp[e.x >> 25];
                const double4 pa = posd[ii], pj = posd[j];
                const double dx = (pa.x - o.x) - pj.x, dy = (pa.y - o.y) - pj.y, dz = (pa.z - oz) - pj.z;
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < pc.rc2) {                     // the exact cutoff, in FP64
                    const double2 lab = __ldg(&lj[d.lj0 + aux[ii].y * d.ntypes + aux[j].y]);
                    const double f = pair_eval_d<EN>(pc, dx, dy, dz, r2, pc.ke * pa.w * pj.w, lab, acc);
                    add_fix2(hx + ii, lx + ii, f * dx);
                    add_fix2(hy + ii, ly + ii, f * dy);
                    add_fix2(hz + ii, lz + ii, f * dz);
                    add_fix2(hx + j, lx + j, -f * dx);
                    add_fix2(hy + j, ly + j, -f * dy);
                    add_fix2(hz + j, lz + j, -f * dz);
                }
            }
            head += n;
            __syncwarp();
        };

        const int gz = wrapi(cz + part, n2);
        for (int c = quarter; c < ncand; c += kF64Split) {
            int ddx, ddy;
            if (part == 0) {
                if (c == 0) { ddx = 0; ddy = 0; }
                else if (c <= sub) { ddx = c; ddy = 0; }
                else { const int u = c - sub - 1; ddx = u % span - sub; ddy = u / span + 1; }
            } else {
                ddx = c % span - sub; ddy = c / span - sub;
            }
            const int g = d.cell0 + wrapi(cx + ddx, n0) + n0 * (wrapi(cy + ddy, n1) + n1 * gz);
            const int j0 = start[g];
            const int nj = count[g];
            const double2 o = offp[c];
            const float xi = pif.x - (float)o.x, yi = pif.y - (float)o.y, zi = pif.z - (float)oz;
            const unsigned code = (unsigned)c << 25;
            // home cell: the atoms after i in cell-sorted order
            const int jmin = (part == 0 && c == 0) ? i0 + lane + 1 : 0;
            for (int j = 0; j < nj; ++j) {
                const float4 pj = posf[j0 + j];
                const float dx = xi - pj.x, dy = yi - pj.y, dz = zi - pj.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const bool hit = vi && r2 < rc2f && __float_as_int(pj.w) != moli && j0 + j >= jmin;
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if (hit)
                    q[(tail + __popc(m & ((1u << lane) - 1u))) & (QCAP - 1)] =
                        make_uint2((unsigned)(j0 + j) | code, (unsigned)lane);
                tail += __popc(m);
                __syncwarp();
                if (tail - head >= 32) eval_round(32);
            }
        }
        if (tail > head) eval_round(tail - head);
    }
    // the warp's record (Ucoul, Ulj, Wc, Wl, W): FP64 warp sums
    double v = 0.0;
    {
        const double uc = warp_sum(acc.uc), ul = warp_sum(acc.ul);
        if (lane == 0) v = uc;
        if (lane == 1) v = ul;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double a = warp_sum(acc.wc[k]), b = warp_sum(acc.wl[k]), t = warp_sum(acc.w[k]);
            if (lane == 2 + k) v = a;
            if (lane == 8 + k) v = b;
            if (lane == 14 + k) v = t;
        }
    }
    if (lane < kPairRec) partial[(size_t)unit * kPairRec + lane] = v;
}

// Opt the pair kernels into their dynamic shared memory (once per context,
// outside any stream capture).
cudaError_t prepare_pair()
{
    cudaError_t e = cudaFuncSetAttribute(k_pair_f64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pair_smem(0));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pair_f64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair_smem(0));
    return e;
}

void launch_pair(const Batch &b, const AtomArrays &a, int precision, const PairConstsF &cf,
                 const PairConstsD &cd, int energy, double *partial, cudaStream_t st)
{
    if (precision == 1) {
        // (item, dz plane) units, kCpWarps per block (item_cap is a multiple of kCpWarps per system)
        const int blocks = b.item_cap * pair_parts(1, b.sub) / kCpWarps;
#define RBSOG_PAIR_CLUSTER(NF, EN)                                                                          \
    k_pair_cluster<NF, EN><<<blocks, 32 * kCpWarps, 0, st>>>(b.sys, b.item_sys, a.items, a.ccl, a.cbox,  \
                                                             a.pos4, a.qt, a.ljf, a.ljf_lo, a.sidx, a.r, \
                                                             b.sub, b.N, b.item_cap, a.ffix, partial, cf)
        // two narrow force Gaussians for Table 2 row 2 (any r_c): unrolled
        if (cf.nff == 2) {
            if (energy) RBSOG_PAIR_CLUSTER(2, true); else RBSOG_PAIR_CLUSTER(2, false);
        } else {
            if (energy) RBSOG_PAIR_CLUSTER(0, true); else RBSOG_PAIR_CLUSTER(0, false);
        }
#undef RBSOG_PAIR_CLUSTER
    } else {
        const int units = b.item_cap * (b.sub + 1) * kF64Split;
        auto k = energy ? k_pair_f64<true> : k_pair_f64<false>;
        k<<<units / kPairWarps, 32 * kPairWarps, pair_smem(0), st>>>(b.sys, b.cell_sys, a.start, a.count, a.items,
                                                                      a.posd, a.posf, a.aux, a.ljd, b.sub, b.N,
                                                                      a.ffix, partial, cd);
    }
}

}  // namespace rbsog
