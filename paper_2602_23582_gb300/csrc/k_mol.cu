// k_mol.cu -- per-molecule terms: harmonic bonds U = k (r - r0)^2, harmonic
// angles U = k (theta - theta0)^2, and the exclusion correction of every
// intramolecular pair: the Fourier part holds each such pair's long-range
// interaction ke q_i q_j F(r) at the minimum image, which is removed:
//   U -= ke q_i q_j F_E(r),  f_i = -ke q_i q_j F~(r) r_ij,  W += f_i (x) r_ij
// (F'(r)/r = -F~(r) for the consistent split w_l = w~_l s~_l^2 / 2, App. C).
//
// One thread per molecule: a molecule's atoms belong to that thread only, so
// forces are added without atomics.  Bonds and angles run in FP64 in both
// builds (few terms; near equilibrium they are small differences of O(1)
// numbers).  In the FP32 build the exclusion terms run in FP32 from FP64
// geometry differences, and the exclusion energy is split as
// -ke q_i q_j F_E(0) (a per-system constant summed on the host in FP64) plus
// ke q_i q_j (F_E(0) - F_E(r)) = ke q_i q_j sum_l w_l (1 - e^{-r^2/s_l^2}),
// evaluated with expm1 so that the FP32 error scales with the small remainder.
#include "internal.h"

namespace rbsog {

namespace {

__device__ __forceinline__ void min_image(double d[3], const double L[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] > 0.5 * L[a]) d[a] -= L[a] * rint(d[a] / L[a]);
        else if (d[a] < -0.5 * L[a]) d[a] -= L[a] * rint(d[a] / L[a]);
    }
}

}  // namespace

// One thread per molecule.  R is the arithmetic type of the terms (float in
// the FP32 build): differences of positions are formed in FP64, then rounded.
template <typename R>
__global__ void __launch_bounds__(kMolChunk)
k_mol(const DevSys *__restrict__ sys, const int *__restrict__ mchunk_sys, const int *__restrict__ mchunk_m0,
      const int *__restrict__ mchunk_n, const int *__restrict__ b_start, const int *__restrict__ a_start,
      const int *__restrict__ e_start, const int *__restrict__ bonds, const double *__restrict__ bk,
      const double *__restrict__ br0, const int *__restrict__ angles, const double *__restrict__ ak,
      const double *__restrict__ at0, const int *__restrict__ excl, const double *__restrict__ r,
      const double *__restrict__ q, double *__restrict__ F /* molecule-term forces */, double *__restrict__ partial,
      const SogConsts sc)
{
    __shared__ double red[15 * (kMolChunk + 1) + 60];
    const int c = blockIdx.x;
    const DevSys &d = sys[mchunk_sys[c]];
    const double L[3] = {d.L[0], d.L[1], d.L[2]};
    double ub = 0, ua = 0, wb[6] = {0, 0, 0, 0, 0, 0};
    R wx[6] = {0, 0, 0, 0, 0, 0};
    R ue_rem = 0;      // sum ke q_i q_j (F_E(0) - F_E(r)) (the constant part is added on the host)
    double ue = 0.0;   // FP64 build: the full exclusion energy
    const int k = threadIdx.x;
    // molecules of the system present (its slot may hold more)
    if (k < min(mchunk_n[c], (d.act ? d.nmol : 0) - (mchunk_m0[c] - d.mol0))) {
        const int mi = mchunk_m0[c] + k;
        // bonds and angles in FP64 in both builds: near equilibrium r - r0 and
        // theta - theta0 are small differences of O(1) numbers, and FP32
        // rounding there would dominate the bonded virial
        for (int e = b_start[mi]; e < b_start[mi + 1]; ++e) {
            const int i = bonds[2 * e], j = bonds[2 * e + 1];
            double dv[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
            min_image(dv, L);
            const double rr = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
            const double dr = rr - br0[e];
            ub += bk[e] * dr * dr;
            const double cf = -2.0 * bk[e] * dr / rr;
            const double f[3] = {cf * dv[0], cf * dv[1], cf * dv[2]};
            for (int a = 0; a < 3; ++a) { F[3 * i + a] += f[a]; F[3 * j + a] -= f[a]; }
            wb[0] += f[0] * dv[0]; wb[1] += f[1] * dv[1]; wb[2] += f[2] * dv[2];
            wb[3] += f[0] * dv[1]; wb[4] += f[0] * dv[2]; wb[5] += f[1] * dv[2];
        }
        for (int e = a_start[mi]; e < a_start[mi + 1]; ++e) {
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
            for (int a = 0; a < 3; ++a) {
                F[3 * i + a] += fi[a];
                F[3 * kk + a] += fk[a];
                F[3 * j + a] -= fi[a] + fk[a];
            }
            wb[0] += fi[0] * d1[0] + fk[0] * d2[0]; wb[1] += fi[1] * d1[1] + fk[1] * d2[1];
            wb[2] += fi[2] * d1[2] + fk[2] * d2[2]; wb[3] += fi[0] * d1[1] + fk[0] * d2[1];
            wb[4] += fi[0] * d1[2] + fk[0] * d2[2]; wb[5] += fi[1] * d1[2] + fk[1] * d2[2];
        }
        for (int e = e_start[mi]; e < e_start[mi + 1]; ++e) {
            const int i = excl[2 * e], j = excl[2 * e + 1];
            double dd[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
            min_image(dd, L);
            const R dv[3] = {(R)dd[0], (R)dd[1], (R)dd[2]};
            const R r2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
            R ft = 0;
            const R qq = (R)(sc.ke * q[i] * q[j]);
            if constexpr (sizeof(R) == 4) {
                // F_E(0) - F_E(r) = sum_l w_l (1 - e^{-r^2/s_l^2}): small, formed without cancellation
                float rem = 0.f;
                for (int l = 0; l < sc.M; ++l) {
                    const float x = (float)r2 / (float)(sc.st[l] * sc.st[l]);
                    const float ex = expf(-x);
                    ft = fmaf((float)sc.wt[l], ex, (float)ft);
                    rem = fmaf((float)sc.w[l], -expm1f(-x), rem);
                }
                for (int l = sc.M; l < sc.ME; ++l)
                    rem = fmaf((float)sc.w[l], -expm1f(-(float)r2 / (float)(sc.s[l] * sc.s[l])), rem);
                ue_rem += qq * (R)rem;
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
            for (int a = 0; a < 3; ++a) { F[3 * i + a] += (double)f[a]; F[3 * j + a] -= (double)f[a]; }
            wx[0] += f[0] * dv[0]; wx[1] += f[1] * dv[1]; wx[2] += f[2] * dv[2];
            wx[3] += f[0] * dv[1]; wx[4] += f[0] * dv[2]; wx[5] += f[1] * dv[2];
        }
    }
    // FP32 build: ue carries the remainder; the host adds -sum ke q_i q_j F_E(0)
    if constexpr (sizeof(R) == 4) ue = (double)ue_rem;
    const double v[15] = {ue, ub, ua, (double)wx[0], (double)wx[1], (double)wx[2],
                          (double)wx[3], (double)wx[4], (double)wx[5], wb[0], wb[1],
                          wb[2], wb[3], wb[4], wb[5]};
    block_reduce_lanes<15, kMolChunk>(v, red, partial + (size_t)c * 15);
}

void launch_mol(const Batch &b, const AtomArrays &a, const MolArrays &m, const SogConsts &sc, double *Fmol,
                double *partial, int precision, cudaStream_t st)
{
    if (m.nmchunks == 0) return;
    if (precision == 1)
        k_mol<float><<<m.nmchunks, kMolChunk, 0, st>>>(b.sys, m.mchunk_sys, m.mchunk_m0, m.mchunk_n, m.b_start,
                                               m.a_start, m.e_start, m.bonds, m.bk, m.br0, m.angles, m.ak,
                                               m.at0, m.excl, a.r, a.q, Fmol, partial, sc);
    else
        k_mol<double><<<m.nmchunks, kMolChunk, 0, st>>>(b.sys, m.mchunk_sys, m.mchunk_m0, m.mchunk_n, m.b_start,
                                                m.a_start, m.e_start, m.bonds, m.bk, m.br0, m.angles, m.ak,
                                                m.at0, m.excl, a.r, a.q, Fmol, partial, sc);
}

}  // namespace rbsog
