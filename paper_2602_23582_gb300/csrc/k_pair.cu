// k_pair.cu -- SOG short-range pair forces, energy and virial over cell lists
// (paper sec. 2.2 and 3.1; eqs. force_SOG, U_short, P_short) plus a 12-6
// Lennard-Jones term cut (unshifted) at r_c.
//
// Per pair with r < r_c and different molecule ids:
//   f   = ke q_i q_j (1/r^3 - sum_{l<M} w~_l e^{-r^2/s~_l^2}) r_vec   (kernel N~)
//   U  += ke q_i q_j (1/r   - sum_{l<ME} w_l e^{-r^2/s_l^2})          (kernel N)
//   W  += f (x) r_vec  (eq. P_short: P^N = W / V)
// Full pairs: each atom sums all its neighbours itself (no atomics, so results
// do not depend on scheduling); energies and virials take half.
//
// Work unit = one warp = a group of up to 32 atoms of one cell (lane = atom,
// in registers) and one dz plane of its neighbour cells (the (2 sub + 1)
// planes of a group run as separate warps, which keeps enough warps in flight;
// their partial forces are summed in a fixed order by the force assembly
// kernel).  The warp walks the (2 sub + 1)^2 neighbour cells of its plane;
// candidate neighbours are read with warp-broadcast loads (every lane the same
// address, served by L1), 32 at a time, and each lane records its hits
// (r^2 < r_c^2, different molecule) in a bit mask, then pushes them, with the
// index of their neighbour cell, into its queue in shared memory.  The warp
// evaluates the SOG kernel in rounds in which every lane with an atom has a
// queued hit, so the expensive part runs with full lanes.  Each block writes
// one record of energy and virial sums (its warps belong to one system).
//
// Coordinates are cell-local.  A neighbour cell's periodic offset d_a w_a is
// split into FP32 hi + lo parts: the cutoff test uses hi, the evaluation
// subtracts both, so that the rounding of w_a does not shift every
// cross-cell distance the same way (a systematic error that the r^-12 and
// 1/r - F(r) terms would amplify).
#include <cuda_fp16.h>

#include "internal.h"

namespace rbsog {

namespace {

constexpr int QCAP = 64;      // FP64 kernel: per-lane queue (power of two); pending <= 32 before a batch
constexpr int kMaxPlane = 32; // neighbour cells of one dz plane (25 for cells of r_c/2)
constexpr int kMaxNb = 128;   // neighbour cells of the stencil (125 for cells of r_c/2)

size_t pair_smem(int precision)
{
    return (size_t)kPairWarps * (QCAP * 32 * sizeof(unsigned) + kMaxPlane * 16);
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

struct AccF {
    float fx, fy, fz;
    float w[6];               // total virial (every step)
    float uc, ul, uq, cuc, cul, cuq;   // energies and sum q_i q_j, with compensation terms
    float wc[6], wl[6];       // Coulomb / LJ split of the virial (energy steps)
};

struct AccD {
    double fx, fy, fz;
    double uc, ul;
    double wc[6], wl[6];
};

// Cutoff decision for a pair close to r_c, in FP64 from the original
// positions with the minimum image, as the CPU reference decides it.
__device__ __forceinline__ bool inside_cutoff_fp64(const double *__restrict__ r, int i, int j, const double L[3],
                                                double rc2)
{
    double r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double dd = r[3 * i + a] - r[3 * j + a];
        dd = L[a] * (dd / L[a] - rint(dd / L[a]));
        r2 += dd * dd;
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

// One pair from the i side.  NF: exponentials of the force kernel (0: pc.nff
// at run time); EN: energies and the Coulomb/LJ virial split.  The force and
// the total virial are computed the same way in both modes.
template <int NF, bool EN>
__device__ __forceinline__ void pair_eval(const PairConstsF &pc, float dx, float dy, float dz, float r2, float qi,
                                          const float2 *__restrict__ ljrow, const float2 *__restrict__ ljlo,
                                          float2 qj, AccF &acc)
{
    float rinv = rsqrt_approx(r2);                       // r^2 of a pair is far above the subnormals
    rinv = rinv * fmaf(-0.5f * r2 * rinv, rinv, 1.5f);   // one Newton step: the approximate
    const float r2inv = rinv * rinv;                     // rsqrt error would bias r^-12 terms
    // force kernel: F~(r) = tail polynomial in r^2 + narrow Gaussians
    float st = pc.tt[kTail];
#pragma unroll
    for (int k = kTail - 1; k >= 0; --k) st = fmaf(st, r2, pc.tt[k]);
    if (NF > 0) {
#pragma unroll
        for (int l = 0; l < NF; ++l) st = fmaf(pc.wt[l], ex2f(-r2 * pc.beta[l]), st);
    } else {
        for (int l = 0; l < pc.nff; ++l) st = fmaf(pc.wt[l], ex2f(-r2 * pc.beta[l]), st);
    }
    const float qq = pc.ke * qi * qj.x;
    const float fc = qq * (r2inv * rinv - st);
    const int tj = __float_as_int(qj.y);
    const float2 lab = ljrow[tj];                        // shared memory
    const float r6inv = r2inv * r2inv * r2inv;
    const float fl = (12.f * lab.x * r6inv - 6.f * lab.y) * r6inv * r2inv;
    const float f = fc + fl;
    acc.fx = fmaf(f, dx, acc.fx);
    acc.fy = fmaf(f, dy, acc.fy);
    acc.fz = fmaf(f, dz, acc.fz);
    const float gx = f * dx, gy = f * dy;
    acc.w[0] = fmaf(gx, dx, acc.w[0]); acc.w[1] = fmaf(gy, dy, acc.w[1]);
    acc.w[2] = fmaf(f * dz, dz, acc.w[2]); acc.w[3] = fmaf(gx, dy, acc.w[3]);
    acc.w[4] = fmaf(gx, dz, acc.w[4]); acc.w[5] = fmaf(gy, dz, acc.w[5]);
    if (EN) {
        // energy kernel N(r) = 1/r - F(r); the constant of the tail is applied
        // to sum q_i q_j in FP64 by the caller
        float se = pc.te[kTail];
#pragma unroll
        for (int k = kTail - 1; k >= 1; --k) se = fmaf(se, r2, pc.te[k]);
        se *= r2;
        for (int l = 0; l < pc.nfe; ++l) {
            const float e = exp2_poly(fmaf(-r2, pc.be_hi[l], -r2 * pc.be_lo[l]));
            se = fmaf(pc.w_hi[l], e, fmaf(pc.w_lo[l], e, se));
        }
        kahan_add(acc.uc, acc.cuc, qq * (rinv - se));
        kahan_add(acc.uq, acc.cuq, qq);
        const float2 lo = ljlo[tj];
        kahan_add(acc.ul, acc.cul, (fmaf(lab.x, r6inv, -lab.y) + fmaf(lo.x, r6inv, -lo.y)) * r6inv);
        const float cx = fc * dx, cy = fc * dy, lx = fl * dx, ly = fl * dy;
        acc.wc[0] = fmaf(cx, dx, acc.wc[0]); acc.wc[1] = fmaf(cy, dy, acc.wc[1]);
        acc.wc[2] = fmaf(fc * dz, dz, acc.wc[2]); acc.wc[3] = fmaf(cx, dy, acc.wc[3]);
        acc.wc[4] = fmaf(cx, dz, acc.wc[4]); acc.wc[5] = fmaf(cy, dz, acc.wc[5]);
        acc.wl[0] = fmaf(lx, dx, acc.wl[0]); acc.wl[1] = fmaf(ly, dy, acc.wl[1]);
        acc.wl[2] = fmaf(fl * dz, dz, acc.wl[2]); acc.wl[3] = fmaf(lx, dy, acc.wl[3]);
        acc.wl[4] = fmaf(lx, dz, acc.wl[4]); acc.wl[5] = fmaf(ly, dz, acc.wl[5]);
    }
}

__device__ __forceinline__ void pair_eval(const PairConstsD &pc, double dx, double dy, double dz, double qi,
                                          const double2 *__restrict__ ljrow, double qj, int tj, AccD &acc)
{
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double rinv = rsqrt(r2);
    const double r2inv = rinv * rinv;
    double st = 0.0, se = 0.0;
    for (int l = 0; l < pc.M; ++l) {
        double e = exp(-r2 * pc.inv_s2[l]);
        st = fma(pc.wt[l], e, st);
        se = fma(pc.w[l], e, se);
    }
    for (int l = pc.M; l < pc.ME; ++l) se = fma(pc.w[l], exp(-r2 * pc.inv_s2[l]), se);
    const double qq = pc.ke * qi * qj;
    const double fc = qq * (r2inv * rinv - st);
    const double ec = qq * (rinv - se);
    const double2 lab = __ldg(&ljrow[tj]);
    const double la = lab.x, lb = lab.y;
    const double r6inv = r2inv * r2inv * r2inv;
    const double fl = (12.0 * la * r6inv - 6.0 * lb) * r6inv * r2inv;
    const double el = (la * r6inv - lb) * r6inv;
    const double f = fc + fl;
    acc.fx = fma(f, dx, acc.fx);
    acc.fy = fma(f, dy, acc.fy);
    acc.fz = fma(f, dz, acc.fz);
    acc.uc += ec;
    acc.ul += el;
    acc.wc[0] += fc * dx * dx; acc.wc[1] += fc * dy * dy; acc.wc[2] += fc * dz * dz;
    acc.wc[3] += fc * dx * dy; acc.wc[4] += fc * dx * dz; acc.wc[5] += fc * dy * dz;
    acc.wl[0] += fl * dx * dx; acc.wl[1] += fl * dy * dy; acc.wl[2] += fl * dz * dz;
    acc.wl[3] += fl * dx * dy; acc.wl[4] += fl * dx * dz; acc.wl[5] += fl * dy * dz;
}

// Next (base, mask) entry of atom ks's hit stream: ep points at it, krem
// entries of plane pl are left; moves to the next plane with entries when
// this one is used up.  The caller asks only for entries that exist.
__device__ __forceinline__ uint2 next_entry(const PairList &L, int ks, int &pl, const uint2 *&ep, int &krem)
{
    while (krem <= 0) {
        ++pl;
        ep = L.ent + (size_t)pl * L.maxent * L.ncap + ks;
        krem = L.nent[pl * L.ncap + ks];
    }
    --krem;
    const uint2 v = *ep;
    ep += L.ncap;
    return v;
}


// Two staged candidates of the list build: (-2 b_x, -2 b_y, -2 b_z, |b|^2) in
// half precision, candidate 2p in the low halves and 2p + 1 in the high ones.
struct __align__(16) HPair {
    __half2 x, y, z, w;
};

__device__ __forceinline__ int wrapi(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

}  // namespace

// ---------------------------------------------------------------------------
// FP32 path in two kernels.
//
// k_pair_build: work unit = 32-atom group x dz plane of its neighbour cells.
// The warp walks the plane's cells in batches of 32 candidates; each lane
// tests its atom against a batch and, when any hit, stores one list entry
// (index of the first candidate | neighbour-cell code << 25, 32-bit hit
// mask) at the next place of its (plane, atom) list.  The lists are laid out
// entry-major over the cell-sorted atoms, ent[(plane * maxent + k) * N + atom],
// so that the 32 lanes of an evaluation warp read entry k of 32 consecutive
// atoms together.
//
// k_pair_eval: one block per 32 consecutive cell-sorted atoms of one system
// (whatever their cells, so the lanes are full); warp k takes segment k of
// kEvalSplit of each atom's hits (all planes in order, split by hit count),
// one hit per lane and round, so every lane carries about the same number of
// pairs, and the block's warps share the same neighbour atoms in L1.
// Segment k writes force partial k, summed in segment order by the force
// assembly.
// ---------------------------------------------------------------------------
// Resident blocks per SM: 20 for one-cell items (80 registers, no spills;
// 32 blocks measured slower), 32 for runs of small cells, whose short units
// need more warps to hide their latency.
template <bool RUNS>
__global__ void __launch_bounds__(32, RUNS ? 32 : 20)
k_pair_build(DevSys *__restrict__ sys, const int *__restrict__ cell_sys, const int *__restrict__ start,
             const int *__restrict__ count, const int2 *__restrict__ items, const float4 *__restrict__ pos4, int sub,
             PairList L, const float rl2_hi)
{
    __shared__ float4 offp[kMaxPlane];                 // x, y offset; column; code of row
    __shared__ HPair cand2[16];
    const int lane = lane_id();
    const int span = 2 * sub + 1;
    const int unit = blockIdx.x;
    const int2 item = items[unit / span];
    if (item.x < 0) return;                            // whole block
    const int part = unit % span;
    const int gc = item.x;
    const int s = cell_sys[gc];
    const DevSys &d = sys[s];
    if (!d.rebuild) return;                            // the system keeps its lists
    // a cell beyond kCellCap atoms (flagged by the scan; e.g. non-finite
    // coordinates all binned into one cell) would make this unit walk
    // millions of candidates: the step is reported failed, skip its pairs
    if (d.flags & FLAG_OVERFLOW) return;
    const int n0 = d.ncell[0], n1 = d.ncell[1], n2 = d.ncell[2];
    const int lc = gc - d.cell0;
    const int cx = lc % n0, cy = (lc / n0) % n1, cz = lc / (n0 * n1);
    const int ddz = part - sub;
    // the item's cells: one cell (group item.y), or a run of rc = -item.y cells
    // of one x-row; a lane's atom lies in cell gc + ldx of the run
    const int rc_n = RUNS && item.y < 0 ? -item.y : 1;
    const int ncol = RUNS ? span + rc_n - 1 : span;    // x columns of the plane's cells
    const int nn = ncol * span;
    for (int nb = lane; nb < nn; nb += 32)
        offp[nb] = make_float4((float)((nb % ncol - sub) * d.w[0]), (float)((nb / ncol - sub) * d.w[1]),
                               __int_as_float(nb % ncol), __int_as_float(part * span * span + (nb / ncol) * span));
    const float ozh = (float)(ddz * d.w[2]);
    __syncwarp();
    int i0, ni;
    if (!RUNS || item.y >= 0) {
        i0 = start[gc] + 32 * item.y;
        ni = min(32, count[gc] - 32 * item.y);
    } else {
        i0 = start[gc];
        ni = start[gc + rc_n - 1] + count[gc + rc_n - 1] - i0;
    }
    const bool vi = lane < ni;
    int ldx = 0;                                       // this lane's cell within the run
    if (RUNS)
        for (int k = 1; k < rc_n; ++k) ldx += (i0 + lane >= start[gc + k]) ? 1 : 0;
    // lanes without an atom sit far away: their cutoff test never passes
    float4 pi = make_float4(1e18f, 1e18f, 1e18f, 0.f);
    if (vi) pi = pos4[i0 + lane];
    int nent = 0, nhit = 0;
    bool overflow = false;
    const int gz = wrapi(cz + ddz, n2);
    // the plane's cells, one per lane: first atom and atom count
    int cj0 = 0, cnj = 0;
    if (lane < nn) {
        const int g = d.cell0 + wrapi(cx + lane % ncol - sub, n0) + n0 * (wrapi(cy + lane / ncol - sub, n1) + n1 * gz);
        cj0 = start[g];
        cnj = count[g];
    }
    // candidates in batches of 32 (one cell at a time), each batch loaded by
    // the whole warp with one coalesced load, one batch ahead, and tested by
    // every lane from shared memory.  The test uses the expanded form
    // |a - b|^2 = |a|^2 + |b|^2 - 2 a.b with a, b relative to the candidate
    // cell's centre: the loading lane stores (-2 b, |b|^2) in half precision,
    // two candidates per half2, so that a pair of candidates costs three
    // packed FMAs and one packed compare.  The test accepts r^2 below
    // 1.025 r_l^2, r_l = r_c + skin the list radius: for the coordinates that
    // occur near r_l (|a| < 2 r_l, |b| < r_l) its rounding error stays below
    // 0.012 r_l^2, inside that margin, and the evaluation decides every pair
    // exactly.  A short batch is padded
    // with entries no lane can hit; pairs of one molecule pass this test and
    // are dropped by the evaluation (a few per atom at most).
    const float hx = 0.5f * (float)d.w[0], hy = 0.5f * (float)d.w[1], hz = 0.5f * (float)d.w[2];
    const float4 far = make_float4(0.f, 0.f, 0.f, 1e30f);
    auto stage = [&](float4 q) {
        const float bx = q.x - hx, by = q.y - hy, bz = q.z - hz;
        return make_float4(-2.f * bx, -2.f * by, -2.f * bz, fmaf(bx, bx, fmaf(by, by, bz * bz)));
    };
    const float rc2_test = 1.025f * rl2_hi;
    int nb = 0, jb = 0, j0 = 0, nj = 0;
    for (;;) {                                         // first non-empty cell (warp-uniform)
        if (nb >= nn) break;
        nj = __shfl_sync(0xffffffffu, cnj, nb);
        if (nj > 0) break;
        ++nb;
    }
    float4 nxt = far;
    if (nb < nn) {
        j0 = __shfl_sync(0xffffffffu, cj0, nb);
        if (lane < nj) nxt = stage(__ldg(pos4 + j0 + lane));
    }
    // this lane's atom relative to the centre of neighbour cell nb is pc - offp[nb]
    // (and its cell lies ldx columns right of the run's first cell)
    const float pcx = pi.x - hx + (float)ldx * (float)d.w[0], pcy = pi.y - hy, pcz = pi.z - hz;
    __half *ch = reinterpret_cast<__half *>(cand2);    // candidate 2p + h: halves h of pair p
    while (nb < nn) {
        const int bnb = nb, bj = j0 + jb;
        {
            const int pp = lane >> 1, h = lane & 1;
            ch[8 * pp + h] = __float2half_rn(nxt.x);
            ch[8 * pp + 2 + h] = __float2half_rn(nxt.y);
            ch[8 * pp + 4 + h] = __float2half_rn(nxt.z);
            ch[8 * pp + 6 + h] = __float2half_rn(nxt.w);
        }
        // advance to the next batch and start its load
        jb += 32;
        if (jb >= nj) {
            jb = 0;
            for (;;) {
                if (++nb >= nn) break;
                nj = __shfl_sync(0xffffffffu, cnj, nb);
                if (nj > 0) break;
            }
            if (nb < nn) j0 = __shfl_sync(0xffffffffu, cj0, nb);
        }
        float4 qn = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool ld = nb < nn && jb + lane < nj;
        if (ld) qn = __ldg(pos4 + j0 + jb + lane);
        __syncwarp();
        const float4 o = offp[bnb];
        const float ax = pcx - o.x, ay = pcy - o.y, az = pcz - ozh;
        // the candidate cell relative to this lane's cell: outside the lane's
        // stencil (a run's far end) it holds no pair within r_c
        const int dxl = __float_as_int(o.z) - ldx;     // sub + x offset of the candidate cell
        const bool incol = !RUNS || (unsigned)dxl < (unsigned)span;
        const __half2 ax2 = __float2half2_rn(ax), ay2 = __float2half2_rn(ay), az2 = __float2half2_rn(az);
        const __half2 thr2 = __float2half2_rn(rc2_test - fmaf(ax, ax, fmaf(ay, ay, az * az)));
        unsigned bits = 0;                             // bit p: candidate 2p, bit 16 + p: candidate 2p + 1
#pragma unroll
        for (int pp = 0; pp < 16; ++pp) {
            const HPair c = cand2[pp];
            const __half2 t = __hfma2(ax2, c.x, __hfma2(ay2, c.y, __hfma2(az2, c.z, c.w)));
            bits |= (__hlt2_mask(t, thr2) & 0x00010001u) << pp;
        }
        // interleave: hit mask bit 2p from bit p, bit 2p + 1 from bit 16 + p
        unsigned lo = bits & 0xffffu, hi = bits >> 16;
        lo = (lo | (lo << 8)) & 0x00ff00ffu; hi = (hi | (hi << 8)) & 0x00ff00ffu;
        lo = (lo | (lo << 4)) & 0x0f0f0f0fu; hi = (hi | (hi << 4)) & 0x0f0f0f0fu;
        lo = (lo | (lo << 2)) & 0x33333333u; hi = (hi | (hi << 2)) & 0x33333333u;
        lo = (lo | (lo << 1)) & 0x55555555u; hi = (hi | (hi << 1)) & 0x55555555u;
        const unsigned hm = incol ? (lo | (hi << 1)) : 0u;   // hits among these 32 candidates
        nxt = ld ? stage(qn) : far;
        __syncwarp();                                  // cand2 is rewritten next round
        const unsigned code = (unsigned)(__float_as_int(o.w) + dxl) << 25;
        // an entry for every batch with a hit, at k = nent of this (plane, atom)
        if (hm != 0u) {
            if (nent < L.maxent) {
                L.ent[((size_t)part * L.maxent + nent) * L.ncap + (i0 + lane)] = make_uint2((unsigned)bj | code, hm);
                ++nent;
                nhit += __popc(hm);
            } else {
                overflow = true;
            }
        }
    }
    if (vi) {
        L.nent[part * L.ncap + i0 + lane] = nent;
        L.nhit[part * L.ncap + i0 + lane] = nhit;
    }
    if (__any_sync(0xffffffffu, overflow) && lane == 0) atomicOr(&sys[s].flags, (int)FLAG_OVERFLOW);
}

template <int NF, bool EN>
__global__ void __launch_bounds__(32 * kEvalSplit * kEvalGroups, (EN ? 4 : 8) / kEvalGroups)
k_pair_eval(const DevSys *__restrict__ sys, const int *__restrict__ item_sys, const float4 *__restrict__ pos4,
            const float2 *__restrict__ qt, const float2 *__restrict__ lj, const float2 *__restrict__ ljlo,
            const int *__restrict__ sidx, const double *__restrict__ r, int sub, int N, const PairList L,
            float4 *__restrict__ Fpart, double *__restrict__ partial, const PairConstsF pc)
{
    __shared__ float4 offh[kMaxNb], offl[kMaxNb];
    __shared__ float2 ljs[EN ? 2 : 1][kMaxTypes * kMaxTypes];   // the system's LJ table (and remainders)
    const int lane = lane_id();
    const int span = 2 * sub + 1;
    // kEvalGroups consecutive groups per block (they share most neighbour
    // atoms in L1), one warp per (group, segment)
    const int warp = threadIdx.x >> 5;
    const int it = blockIdx.x * kEvalGroups + warp / kEvalSplit, seg = warp % kEvalSplit;
    // the block's groups lie in one system (item_cap per system is a multiple of kEvalGroups)
    const DevSys &d = sys[item_sys[it]];
    // evaluation group: 32 consecutive cell-sorted atoms of one system (group
    // g of the system uses the record slots of its work item item0 + g)
    const int g32 = 32 * (it - d.item0), nlive = live_n(d);
    double u0 = 0.0, u1 = 0.0;
    float wv[18];                                      // Wc, Wl (energy steps), W
#pragma unroll
    for (int k = 0; k < 18; ++k) wv[k] = 0.f;
    const bool ok = !(d.flags & FLAG_OVERFLOW);       // lists of a failed step are not walked
    if (ok && 32 * (blockIdx.x * kEvalGroups - d.item0) < nlive) {   // block-uniform: some group is live
        // neighbour-cell offsets d_a w_a as FP32 hi + lo (the rounding of w
        // must not shift every cross-cell distance the same way)
        for (int nb = threadIdx.x; nb < span * span * span; nb += blockDim.x) {
            const double ox = (nb % span - sub) * d.w[0], oy = ((nb / span) % span - sub) * d.w[1],
                         oz = (nb / (span * span) - sub) * d.w[2];
            const float hx = (float)ox, hy = (float)oy, hz = (float)oz;
            offh[nb] = make_float4(hx, hy, hz, 0.f);
            offl[nb] = make_float4((float)(ox - (double)hx), (float)(oy - (double)hy), (float)(oz - (double)hz), 0.f);
        }
        for (int t = threadIdx.x; t < d.ntypes * d.ntypes; t += blockDim.x) {
            ljs[0][t] = lj[d.lj0 + t];
            if (EN) ljs[EN ? 1 : 0][t] = ljlo[d.lj0 + t];
        }
        __syncthreads();
    }
    if (ok && g32 < nlive) {                           // warp-uniform
        const int ks = d.atom0 + g32 + lane;           // this lane's atom (cell-sorted index)
        const bool vi = g32 + lane < nlive;
        float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 pq = make_float2(0.f, 0.f);
        // this warp takes hits [h0, h1) of the lane's stream (all planes in order)
        int nh = 0, pl = 0, krem = 0;
        const uint2 *ep = L.ent + ks;
        unsigned base = 0u, mask = 0u;
        if (vi) {
            pi = pos4[ks];
            pq = qt[ks];
            int tot = 0;
            for (int p2 = 0; p2 < span; ++p2) tot += L.nhit[p2 * L.ncap + ks];
            const int h0 = (int)((long long)tot * seg / kEvalSplit);
            const int h1 = (int)((long long)tot * (seg + 1) / kEvalSplit);
            nh = h1 - h0;
            if (nh > 0) {
                int skip = h0;
                int hp = L.nhit[ks];
                while (skip >= hp) { skip -= hp; ++pl; hp = L.nhit[pl * L.ncap + ks]; }
                ep = L.ent + (size_t)pl * L.maxent * L.ncap + ks;
                krem = L.nent[pl * L.ncap + ks];
                while (skip > 0) {                     // walk entries up to hit h0
                    const uint2 en = *ep;
                    ep += L.ncap;
                    --krem;
                    const int cc = __popc(en.y);
                    if (cc <= skip) {
                        skip -= cc;
                    } else {
                        base = en.x;
                        mask = en.y;
                        for (; skip > 0; --skip) mask &= mask - 1u;
                    }
                }
            }
        }
        const int rowi = __float_as_int(pq.y) * d.ntypes;
        const float2 *ljrow = ljs[0] + rowi, *ljlorow = ljs[EN ? 1 : 0] + rowi;
        AccF acc;
        acc.fx = acc.fy = acc.fz = 0.f;
        acc.uc = acc.ul = acc.uq = acc.cuc = acc.cul = acc.cuq = 0.f;
#pragma unroll
        for (int k = 0; k < 6; ++k) acc.w[k] = acc.wc[k] = acc.wl[k] = 0.f;
        // one hit ahead: the next hit's atom data, and the next list entry once
        // the current one has started, are loaded while this hit is evaluated
        int left = nh;                                 // hits of this lane still to evaluate
        if (left > 0 && mask == 0u) {
            const uint2 en = next_entry(L, ks, pl, ep, krem);
            base = en.x;
            mask = en.y;
        }
        uint2 nxt = make_uint2(0u, 0u);
        if (left > __popc(mask)) nxt = next_entry(L, ks, pl, ep, krem);
        unsigned e = 0u;
        float4 pj = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 qj = make_float2(0.f, 0.f);
        if (left > 0) {
            e = base + (unsigned)(__ffs(mask) - 1);
            mask &= mask - 1u;
            pj = pos4[e & 0x1ffffffu];
            qj = qt[e & 0x1ffffffu];
        }
        const int tmax = __reduce_max_sync(0xffffffffu, nh);
        for (int kk = 0; kk < tmax; ++kk) {
            if (kk < nh) {
                const unsigned ec = e;
                const float4 pjc = pj;
                const float2 qjc = qj;
                if (--left > 0) {
                    if (mask == 0u) {
                        base = nxt.x;
                        mask = nxt.y;
                        if (left > __popc(mask)) nxt = next_entry(L, ks, pl, ep, krem);
                    }
                    e = base + (unsigned)(__ffs(mask) - 1);
                    mask &= mask - 1u;
                    pj = pos4[e & 0x1ffffffu];
                    qj = qt[e & 0x1ffffffu];
                }
                const float4 oh = offh[ec >> 25], ol = offl[ec >> 25];
                const float dx = ((pi.x - oh.x) - pjc.x) - ol.x, dy = ((pi.y - oh.y) - pjc.y) - ol.y,
                            dz = ((pi.z - oh.z) - pjc.z) - ol.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                // pairs within a relative 1e-5 of r_c^2 are decided in FP64 from the
                // original positions (the energy kernel N is about 2e-3 / A at r_c,
                // so one pair on the wrong side shifts U by ~ke q_i q_j 2e-3)
                if (__float_as_int(pjc.w) != __float_as_int(pi.w) &&   // not of one molecule
                    (r2 < pc.rc2_lo || (r2 < pc.rc2_hi &&
                     inside_cutoff_fp64(r, sidx[ks], sidx[ec & 0x1ffffffu], d.L, pc.rc2d))))
                    pair_eval<NF, EN>(pc, dx, dy, dz, r2, pq.x, ljrow, ljlorow, qjc, acc);
            }
        }
        if (vi) Fpart[(size_t)seg * N + ks] = make_float4(acc.fx, acc.fy, acc.fz, 0.f);
        // virials: FP32 warp sums; energies: FP64 (compensated lanes), with the
        // constant of the energy tail applied to sum q_i q_j here
#pragma unroll
        for (int k = 0; k < 6; ++k) wv[12 + k] = warp_sumf(acc.w[k]);
        if (EN) {
            u0 = warp_sum((double)acc.uc - (double)acc.cuc - pc.te0 * ((double)acc.uq - (double)acc.cuq));
            u1 = warp_sum((double)acc.ul - (double)acc.cul);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                wv[k] = warp_sumf(acc.wc[k]);
                wv[6 + k] = warp_sumf(acc.wl[k]);
            }
        }
    }
    // one record per (item, segment): lane t writes value t (each pair was seen from both atoms)
    double v = 0.0;
    if (lane == 0) v = u0;
    if (lane == 1) v = u1;
#pragma unroll
    for (int k = 0; k < 18; ++k)
        if (lane == 2 + k) v = (double)wv[k];
    if (lane < kPairRec) partial[((size_t)it * kEvalSplit + seg) * kPairRec + lane] = 0.5 * v;
}

// ---------------------------------------------------------------------------
// FP64 kernel (same structure; plane offsets in FP64 need no lo part)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * kPairWarps)
k_pair_f64(const DevSys *__restrict__ sys, const int *__restrict__ cell_sys, const int *__restrict__ start,
           const int *__restrict__ count, const int2 *__restrict__ items, const double4 *__restrict__ posd,
           const int2 *__restrict__ aux, const double2 *__restrict__ lj, int sub, int N,
           double4 *__restrict__ Fpart, double *__restrict__ partial, const PairConstsD pc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double rec[kPairWarps][kPairRec];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    unsigned *q = reinterpret_cast<unsigned *>(smem) + warp * QCAP * 32;
    double2 *offp = reinterpret_cast<double2 *>(smem + kPairWarps * QCAP * 32 * sizeof(unsigned)) + warp * kMaxPlane;
    const int span = 2 * sub + 1;
    // unit = (work item, dz plane, quarter): the quarter takes every kF64Split-th
    // cell of the plane, so that small systems still fill the SMs' FP64 pipes
    const int unit = blockIdx.x * kPairWarps + warp;
    const int2 item = items[unit / (span * kF64Split)];
    const int part = (unit / kF64Split) % span, quarter = unit % kF64Split;
    double red[kPairRec];
#pragma unroll
    for (int k = 0; k < kPairRec; ++k) red[k] = 0.0;
    // (a system with a cell beyond kCellCap atoms has failed its step: skipped)
    if (item.x >= 0 && !(sys[cell_sys[item.x]].flags & FLAG_OVERFLOW)) {
        const int gc = item.x;
        const DevSys &d = sys[cell_sys[gc]];
        const int n0 = d.ncell[0], n1 = d.ncell[1], n2 = d.ncell[2];
        const int lc = gc - d.cell0;
        const int cx = lc % n0, cy = (lc / n0) % n1, cz = lc / (n0 * n1);
        const int ddz = part - sub;
        const double oz = ddz * d.w[2];
        for (int nb = lane; nb < span * span; nb += 32)
            offp[nb] = make_double2((nb % span - sub) * d.w[0], (nb / span - sub) * d.w[1]);
        __syncwarp();
        const int i0 = start[gc] + 32 * item.y;
        const int ni = min(32, count[gc] - 32 * item.y);
        const bool vi = lane < ni;
        double4 pi = make_double4(0, 0, 0, 0);
        int2 ai = make_int2(-0x7fffffff, 0);
        if (vi) { pi = posd[i0 + lane]; ai = aux[i0 + lane]; }
        const double2 *ljrow = lj + d.lj0 + ai.y * d.ntypes;
        const double rc2 = pc.rc2;
        AccD acc;
        acc.fx = acc.fy = acc.fz = 0.0;
        acc.uc = acc.ul = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) acc.wc[k] = acc.wl[k] = 0.0;
        int head = 0, tail = 0;

        auto eval_one = [&](unsigned e) {
            const unsigned j = e & 0x1ffffffu;
            const double4 pj = posd[j];
            const int tj = aux[j].y;
            const double2 o = offp[e >> 25];
            pair_eval(pc, (pi.x - o.x) - pj.x, (pi.y - o.y) - pj.y, (pi.z - oz) - pj.z, pi.w, ljrow, pj.w, tj, acc);
        };
        auto pop = [&]() {
            const int slot = (head & (QCAP - 1)) * 32 + lane;
            ++head;
            eval_one(q[slot]);
        };

        const int gz = wrapi(cz + ddz, n2);
        for (int nb = quarter; nb < span * span; nb += kF64Split) {
            const int g = d.cell0 + wrapi(cx + nb % span - sub, n0) + n0 * (wrapi(cy + nb / span - sub, n1) + n1 * gz);
            const int j0 = start[g], nj = count[g];
            const double2 o = offp[nb];
            const double xi = pi.x - o.x, yi = pi.y - o.y, zi = pi.z - oz;
            const unsigned code = (unsigned)nb << 25;
            for (int jb = 0; jb < nj; jb += 32) {
                const int je = min(jb + 32, nj);
                for (int j = jb; j < je; ++j) {
                    const double4 pj = posd[j0 + j];
                    const double dx = xi - pj.x, dy = yi - pj.y, dz = zi - pj.z;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (vi && r2 < rc2 && aux[j0 + j].x != ai.x) {
                        q[(tail & (QCAP - 1)) * 32 + lane] = (unsigned)(j0 + j) | code;
                        ++tail;
                    }
                }
                const int mn = __reduce_min_sync(0xffffffffu, vi ? tail - head : QCAP);
                for (int t = 0; t < mn; ++t)
                    if (vi) pop();
                while (__reduce_max_sync(0xffffffffu, tail - head) > QCAP - 32)
                    if (tail > head) pop();
            }
        }
        while (__any_sync(0xffffffffu, tail > head))
            if (tail > head) pop();
        if (vi) Fpart[(size_t)(part * kF64Split + quarter) * N + i0 + lane] = make_double4(acc.fx, acc.fy, acc.fz, 0.0);
        const double v[14] = {acc.uc, acc.ul, acc.wc[0], acc.wc[1], acc.wc[2], acc.wc[3], acc.wc[4],
                              acc.wc[5], acc.wl[0], acc.wl[1], acc.wl[2], acc.wl[3], acc.wl[4], acc.wl[5]};
#pragma unroll
        for (int k = 0; k < 14; ++k) red[k] = warp_sum(v[k]);
#pragma unroll
        for (int k = 0; k < 6; ++k) red[14 + k] = red[2 + k] + red[8 + k];
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kPairRec; ++k) rec[warp][k] = red[k];
    }
    __syncthreads();
    if (threadIdx.x < kPairRec) {
        const int t = threadIdx.x;
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kPairWarps; ++w) s += rec[w][t];
        partial[(size_t)blockIdx.x * kPairRec + t] = 0.5 * s;
    }
}

// Opt the pair kernels into their dynamic shared memory (once per context,
// outside any stream capture).
cudaError_t prepare_pair()
{
    return cudaFuncSetAttribute(k_pair_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair_smem(0));
}

void launch_pair(const Batch &b, const AtomArrays &a, int precision, const PairConstsF &cf,
                 const PairConstsD &cd, int energy, double *partial, cudaStream_t st)
{
    // item_cap is a multiple of kItemAlign per system, so every block lies in one system
    const int units = b.item_cap * (2 * b.sub + 1);
    if (precision == 1) {
        // runs of several cells per item occur with cells of r_c / 2 (a dozen atoms)
        auto build = b.sub >= 2 ? k_pair_build<true> : k_pair_build<false>;
        build<<<units, 32, 0, st>>>(b.sys, b.cell_sys, a.start, a.count, a.items, a.pos4, b.sub, a.plist, cf.rl2_hi);
#define RBSOG_PAIR_EVAL(NF, EN)                                                                                  \
    k_pair_eval<NF, EN><<<b.item_cap / kEvalGroups, 32 * kEvalSplit * kEvalGroups, 0, st>>>(b.sys, b.item_sys, \
                                                                a.pos4, a.qt, a.ljf, a.ljf_lo, a.sidx, a.r, b.sub, \
                                                                b.N, a.plist, a.fpart4, partial, cf)
        if (cf.nff == 4) {
            if (energy) RBSOG_PAIR_EVAL(4, true); else RBSOG_PAIR_EVAL(4, false);
        } else {
            if (energy) RBSOG_PAIR_EVAL(0, true); else RBSOG_PAIR_EVAL(0, false);
        }
#undef RBSOG_PAIR_EVAL
    } else {
        k_pair_f64<<<units * kF64Split / kPairWarps, 32 * kPairWarps, pair_smem(0), st>>>(
            b.sys, b.cell_sys, a.start, a.count, a.items, a.posd, a.aux, a.ljd, b.sub, b.N, a.fpartd, partial, cd);
    }
}

}  // namespace rbsog
