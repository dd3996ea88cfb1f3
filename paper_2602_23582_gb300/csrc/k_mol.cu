// k_mol.cu -- per-molecule terms: harmonic bonds U = k (r - r0)^2, harmonic
// angles U = k (theta - theta0)^2, and the exclusion correction of every
// intramolecular pair: the Fourier part holds each such pair's long-range
// interaction ke q_i q_j F(r) at the minimum image, which is removed:
//   U -= ke q_i q_j F_E(r),  f_i = -ke q_i q_j F~(r) r_ij,  W += f_i (x) r_ij
// (F'(r)/r = -F~(r) for the consistent split w_l = w~_l s~_l^2 / 2, App. C).
//
// One warp per molecule, its terms spread over the lanes (see k_mol); every
// sum runs in a fixed order, so results do not depend on scheduling.  Bonds
// and angles run in FP64 in both builds (few terms; near equilibrium they
// are small differences of O(1) numbers).  In the FP32 build the exclusion terms run in FP32 from FP64
// geometry differences, and the exclusion energy is split as
// -ke q_i q_j F_E(0) (a per-system constant summed on the host in FP64) plus
// ke q_i q_j (F_E(0) - F_E(r)) = ke q_i q_j sum_l w_l (1 - e^{-r^2/s_l^2}),
// evaluated with expm1 so that the FP32 error scales with the small remainder.
#include "internal.h"

namespace rbsog {

namespace {

// the box of a system in registers: edges, tilts (xy, xz, yz), tilted or not
struct Box {
    double L[3], t[3];
    bool tri;
};

__device__ __forceinline__ void min_image(double d[3], const Box &B)
{
    if (B.tri) {
        // the image whose fractional components s = h^{-1} d lie in [-1/2, 1/2]
        // (h upper triangular: back substitution), d <- d - h rint(s)
        const double s2 = d[2] / B.L[2];
        const double s1 = (d[1] - B.t[2] * s2) / B.L[1];
        const double s0 = (d[0] - B.t[0] * s1 - B.t[1] * s2) / B.L[0];
        const double n0 = rint(s0), n1 = rint(s1), n2 = rint(s2);
        d[0] -= B.L[0] * n0 + B.t[0] * n1 + B.t[1] * n2;
        d[1] -= B.L[1] * n1 + B.t[2] * n2;
        d[2] -= B.L[2] * n2;
        return;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] > 0.5 * B.L[a]) d[a] -= B.L[a] * rint(d[a] / B.L[a]);
        else if (d[a] < -0.5 * B.L[a]) d[a] -= B.L[a] * rint(d[a] / B.L[a]);
    }
}

// Contributions of one term to the forces of its atoms (at most 3).
struct TermF {
    int n;
    int atom[3];
    double f[3][3];
};

// Bond e: U = k (r - r0)^2 in FP64 (near equilibrium r - r0 is a small
// difference of O(1) numbers; FP32 rounding there would dominate the bonded
// virial).
__device__ __forceinline__ void bond_term(int e, const int *__restrict__ bonds, const double *__restrict__ bk,
                                          const double *__restrict__ br0, const double *__restrict__ r,
                                          const Box &L, double &ub, double wb[6], TermF &t)
{
    const int i = bonds[2 * e], j = bonds[2 * e + 1];
    double dv[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
    min_image(dv, L);
    const double rr = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    const double dr = rr - br0[e];
    ub += bk[e] * dr * dr;
    const double cf = -2.0 * bk[e] * dr / rr;
    const double f[3] = {cf * dv[0], cf * dv[1], cf * dv[2]};
    t.n = 2;
    t.atom[0] = i; t.atom[1] = j;
    for (int a = 0; a < 3; ++a) { t.f[0][a] = f[a]; t.f[1][a] = -f[a]; }
    wb[0] += f[0] * dv[0]; wb[1] += f[1] * dv[1]; wb[2] += f[2] * dv[2];
    wb[3] += f[0] * dv[1]; wb[4] += f[0] * dv[2]; wb[5] += f[1] * dv[2];
}

// Angle e (i, j at the vertex, k): U = k (theta - theta0)^2 in FP64.
__device__ __forceinline__ void angle_term(int e, const int *__restrict__ angles, const double *__restrict__ ak,
                                           const double *__restrict__ at0, const double *__restrict__ r,
                                           const Box &L, double &ua, double wb[6], TermF &t)
{
    const int i = angles[3 * e], j = angles[3 * e + 1], kk = angles[3 * e + 2];
    double d1[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
    double d2[3] = {r[3 * kk] - r[3 * j], r[3 * kk + 1] - r[3 * j + 1], r[3 * kk + 2] - r[3 * j + 2]};
    min_image(d1, L);
    min_image(d2, L);
    const double r1 = sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
    const double r2 = sqrt(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
    double cs = (d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2]) / (r1 * r2);
    cs = cs > 1.0 ? 1.0 : (cs < -1.0 ? -1.0 : cs);
    const double th = acos(cs);
    double sn = sqrt(1.0 - cs * cs);
    if (sn < 1e-12) sn = 1e-12;
    const double dth = th - at0[e];
    ua += ak[e] * dth * dth;
    const double g = 2.0 * ak[e] * dth / sn;
    double fi[3], fk[3];
    for (int a = 0; a < 3; ++a) {
        fi[a] = g * (d2[a] / (r1 * r2) - cs * d1[a] / (r1 * r1));
        fk[a] = g * (d1[a] / (r1 * r2) - cs * d2[a] / (r2 * r2));
    }
    t.n = 3;
    t.atom[0] = i; t.atom[1] = kk; t.atom[2] = j;
    for (int a = 0; a < 3; ++a) { t.f[0][a] = fi[a]; t.f[1][a] = fk[a]; t.f[2][a] = -(fi[a] + fk[a]); }
    wb[0] += fi[0] * d1[0] + fk[0] * d2[0]; wb[1] += fi[1] * d1[1] + fk[1] * d2[1];
    wb[2] += fi[2] * d1[2] + fk[2] * d2[2]; wb[3] += fi[0] * d1[1] + fk[0] * d2[1];
    wb[4] += fi[0] * d1[2] + fk[0] * d2[2]; wb[5] += fi[1] * d1[2] + fk[1] * d2[2];
}

// Exclusion e: removes the pair's Fourier-part interaction (see the header).
template <typename R>
__device__ __forceinline__ void excl_term(int e, const int *__restrict__ excl, const double *__restrict__ r,
                                          const double *__restrict__ q, const Box &L, const SogConsts &sc,
                                          int en, R &ue_rem, double &ue, R wx[6], TermF &t)
{
    const int i = excl[2 * e], j = excl[2 * e + 1];
    double dd[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
    min_image(dd, L);
    const R dv[3] = {(R)dd[0], (R)dd[1], (R)dd[2]};
    const R r2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
    R ft = 0;
    const R qq = (R)(sc.ke * q[i] * q[j]);
    if constexpr (sizeof(R) == 4) {
        // F_E(0) - F_E(r) = sum_l w_l (1 - e^{-r^2/s_l^2}): small, formed without cancellation
        // FP32 constants only: no FP64 operation or conversion per term; the
        // energy remainder only on energy steps (en)
        for (int l = 0; l < sc.M; ++l) ft = fmaf(sc.wtf[l], expf(-(float)r2 * sc.ist2f[l]), (float)ft);
        if (en) {
            float rem = 0.f;
            for (int l = 0; l < sc.ME; ++l) rem = fmaf(sc.wf[l], -expm1f(-(float)r2 * sc.is2f[l]), rem);
            ue_rem += qq * (R)rem;
        }
    } else {
        double fe = 0.0, ftd = 0.0;
        for (int l = 0; l < sc.M; ++l) {
            const double ex = exp(-(double)r2 / (sc.st[l] * sc.st[l]));
            ftd += sc.wt[l] * ex;
            fe += sc.w[l] * ex;
        }
        for (int l = sc.M; l < sc.ME; ++l) fe += sc.w[l] * exp(-(double)r2 / (sc.s[l] * sc.s[l]));
        ft = (R)ftd;
        ue -= sc.ke * q[i] * q[j] * fe;
    }
    const R f[3] = {-qq * ft * dv[0], -qq * ft * dv[1], -qq * ft * dv[2]};
    t.n = 2;
    t.atom[0] = i; t.atom[1] = j;
    for (int a = 0; a < 3; ++a) { t.f[0][a] = (double)f[a]; t.f[1][a] = -(double)f[a]; }
    wx[0] += f[0] * dv[0]; wx[1] += f[1] * dv[1]; wx[2] += f[2] * dv[2];
    wx[3] += f[0] * dv[1]; wx[4] += f[0] * dv[2]; wx[5] += f[1] * dv[2];
}

}  // namespace

// A block takes the molecules of a chunk (kMolChunk of them for systems of
// small molecules, kMolChunkLarge otherwise; at most one per thread).  A molecule with at most
// kSmallTerms terms is one thread's (its terms in order: bonds, angles,
// exclusions, each added to its atoms' forces at once).  A larger molecule is
// one warp's: its terms are spread over the lanes in passes of kTermPass,
// each term stores its atoms' contributions in shared memory (in R), and
// lane k sums the contributions to the pass's k-th atom in term order and
// adds the sum to F.  F is zeroed by the caller; a molecule's atoms
// are written by its thread or warp only, and every sum runs in a fixed
// order.  R is the arithmetic type of the exclusion terms (float in the FP32
// build): differences of positions are formed in FP64, then rounded.
constexpr int kMolWarps = 4, kTermPass = 64;

template <typename R>
__global__ void __launch_bounds__(32 * kMolWarps)
k_mol(const DevSys *__restrict__ sys, const int *__restrict__ mchunk_sys, const int *__restrict__ mchunk_m0,
      const int *__restrict__ mchunk_n, const int *__restrict__ b_start, const int *__restrict__ a_start,
      const int *__restrict__ e_start, const int *__restrict__ bonds, const double *__restrict__ bk,
      const double *__restrict__ br0, const int *__restrict__ angles, const double *__restrict__ ak,
      const double *__restrict__ at0, const int *__restrict__ excl, const double *__restrict__ r,
      const double *__restrict__ q, double *__restrict__ F /* molecule-term forces */, double *__restrict__ partial,
      const SogConsts sc, int en)
{
    static_assert(32 * kMolWarps >= kMolChunk, "one thread per molecule of a chunk");
    constexpr int NT = 32 * kMolWarps, NS = 3 * kTermPass;
    __shared__ double red[15 * (NT + 1) + 60];
    __shared__ int s_atom[kMolWarps][NS];
    __shared__ R s_f[kMolWarps][NS][3];         // contributions in R: FP32 adds in the FP32 build
    const int c = blockIdx.x, w = threadIdx.x >> 5, lane = lane_id();
    const DevSys &d = sys[mchunk_sys[c]];
    const Box L = {{d.L[0], d.L[1], d.L[2]}, {d.tilt[0], d.tilt[1], d.tilt[2]}, d.tri != 0};
    double ub = 0, ua = 0, wb[6] = {0, 0, 0, 0, 0, 0};
    R wx[6] = {0, 0, 0, 0, 0, 0};
    R ue_rem = 0;      // sum ke q_i q_j (F_E(0) - F_E(r)) (the constant part is added on the host)
    double ue = 0.0;   // FP64 build: the full exclusion energy
    // molecules of the system present (its slot may hold more)
    const int nm = min(mchunk_n[c], (d.act ? d.nmol : 0) - (mchunk_m0[c] - d.mol0));
    const int m0 = mchunk_m0[c];
    // small molecules: one thread each
    if ((int)threadIdx.x < nm) {
        const int mi = m0 + threadIdx.x;
        const int b0 = b_start[mi], nb = b_start[mi + 1] - b0;
        const int a0 = a_start[mi], na = a_start[mi + 1] - a0;
        const int e0 = e_start[mi], ne = e_start[mi + 1] - e0;
        if (nb + na + ne <= kSmallTerms) {
            for (int t = 0; t < nb + na + ne; ++t) {
                TermF tf;
                if (t < nb) bond_term(b0 + t, bonds, bk, br0, r, L, ub, wb, tf);
                else if (t < nb + na) angle_term(a0 + t - nb, angles, ak, at0, r, L, ua, wb, tf);
                else excl_term<R>(e0 + t - nb - na, excl, r, q, L, sc, en, ue_rem, ue, wx, tf);
                for (int v = 0; v < tf.n; ++v)
                    for (int x = 0; x < 3; ++x) F[3 * tf.atom[v] + x] += tf.f[v][x];
            }
        }
    }
    // large molecules: one warp each, in chunk order over the warps
    int *sa = s_atom[w];
    R (*sf)[3] = s_f[w];
    int big = 0;                                       // large molecules seen so far (warp-uniform)
    for (int k = 0; k < nm; ++k) {
        const int mi = m0 + k;
        const int b0 = b_start[mi], nb = b_start[mi + 1] - b0;
        const int a0 = a_start[mi], na = a_start[mi + 1] - a0;
        const int e0 = e_start[mi], ne = e_start[mi + 1] - e0;
        const int nt = nb + na + ne;
        if (nt <= kSmallTerms) continue;
        if (big++ % kMolWarps != w) continue;
        for (int p0 = 0; p0 < nt; p0 += kTermPass) {
            const int np = min(kTermPass, nt - p0);
            for (int u = lane; u < kTermPass; u += 32) {
                const int t = p0 + u;
                TermF tf;
                tf.n = 0;
                if (u < np) {
                    if (t < nb) bond_term(b0 + t, bonds, bk, br0, r, L, ub, wb, tf);
                    else if (t < nb + na) angle_term(a0 + t - nb, angles, ak, at0, r, L, ua, wb, tf);
                    else excl_term<R>(e0 + t - nb - na, excl, r, q, L, sc, en, ue_rem, ue, wx, tf);
                }
                for (int v = 0; v < 3; ++v) {
                    sa[3 * u + v] = v < tf.n ? tf.atom[v] : -1;
                    if (v < tf.n)
                        for (int x = 0; x < 3; ++x) sf[3 * u + v][x] = (R)tf.f[v][x];
                }
            }
            __syncwarp();
            // per atom (a molecule's atoms are contiguous): lane k takes atom
            // lo + k of the pass and sums its slots in slot order; every lane
            // reads the same slot at a time (a shared-memory broadcast), so
            // the scans run side by side
            int lo = 0x7fffffff, hi = -1;
            for (int sl = lane; sl < 3 * np; sl += 32) {
                const int at = sa[sl];
                if (at >= 0) { lo = min(lo, at); hi = max(hi, at); }
            }
            lo = __reduce_min_sync(0xffffffffu, lo);
            hi = __reduce_max_sync(0xffffffffu, hi);
            for (int at = lo + lane; at <= hi; at += 32) {
                // the adds run in R: in the FP32 build no FP64 instruction is
                // issued here, where few lanes are active (an FP64 warp
                // instruction costs the same for one lane as for 32)
                R g[3] = {0, 0, 0};
                bool any = false;
                for (int u = 0; u < 3 * np; ++u) {
                    if (sa[u] != at) continue;
                    if (any) {
                        g[0] += sf[u][0]; g[1] += sf[u][1]; g[2] += sf[u][2];
                    } else {
                        g[0] = sf[u][0]; g[1] = sf[u][1]; g[2] = sf[u][2];
                        any = true;
                    }
                }
                if (!any) continue;
                const double gd[3] = {(double)g[0], (double)g[1], (double)g[2]};
                const double f0 = F[3 * at], f1 = F[3 * at + 1], f2 = F[3 * at + 2];
                F[3 * at] = f0 + gd[0];
                F[3 * at + 1] = f1 + gd[1];
                F[3 * at + 2] = f2 + gd[2];
            }
            __syncwarp();
        }
    }
    // FP32 build: ue carries the remainder; the host adds -sum ke q_i q_j F_E(0)
    if constexpr (sizeof(R) == 4) ue = (double)ue_rem;
    const double v[15] = {ue, ub, ua, (double)wx[0], (double)wx[1], (double)wx[2],
                          (double)wx[3], (double)wx[4], (double)wx[5], wb[0], wb[1],
                          wb[2], wb[3], wb[4], wb[5]};
    block_reduce_lanes<15, NT>(v, red, partial + (size_t)c * 15);
}

void launch_mol(const Batch &b, const AtomArrays &a, const MolArrays &m, const SogConsts &sc, double *Fmol,
                double *partial, int precision, int energy, cudaStream_t st)
{
    if (m.nmchunks == 0) return;
    if (precision == 1)
        k_mol<float><<<m.nmchunks, 32 * kMolWarps, 0, st>>>(b.sys, m.mchunk_sys, m.mchunk_m0, m.mchunk_n, m.b_start,
                                               m.a_start, m.e_start, m.bonds, m.bk, m.br0, m.angles, m.ak,
                                               m.at0, m.excl, a.r, a.q, Fmol, partial, sc, energy);
    else
        k_mol<double><<<m.nmchunks, 32 * kMolWarps, 0, st>>>(b.sys, m.mchunk_sys, m.mchunk_m0, m.mchunk_n, m.b_start,
                                                m.a_start, m.e_start, m.bonds, m.bk, m.br0, m.angles, m.ak,
                                                m.at0, m.excl, a.r, a.q, Fmol, partial, sc, energy);
}

}  // namespace rbsog
