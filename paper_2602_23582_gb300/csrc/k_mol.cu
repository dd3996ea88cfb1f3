// k_mol.cu -- per-molecule terms: harmonic bonds U = k (r - r0)^2, harmonic
// angles U = k (theta - theta0)^2, and the exclusion correction of every
// intramolecular pair: the Fourier part holds each such pair's long-range
// interaction ke q_i q_j F(r) at the minimum image, which is removed:
//   U -= ke q_i q_j F_E(r),  f_i = -ke q_i q_j F~(r) r_ij,  W += f_i (x) r_ij
// (F'(r)/r = -F~(r) for the consistent split w_l = w~_l s~_l^2 / 2, App. C).
//
// One thread per molecule: a molecule's atoms belong to that thread only, so
// forces are added without atomics.  Geometry differences are formed in FP64;
// in the FP32 build the Gaussians of the exclusion term run in FP32.
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

template <bool F32>
__global__ void __launch_bounds__(128)
k_mol(const DevSys *__restrict__ sys, const int *__restrict__ mchunk_sys, const int *__restrict__ mchunk_m0,
      const int *__restrict__ mchunk_n, const int *__restrict__ b_start, const int *__restrict__ a_start,
      const int *__restrict__ e_start, const int *__restrict__ bonds, const double *__restrict__ bk,
      const double *__restrict__ br0, const int *__restrict__ angles, const double *__restrict__ ak,
      const double *__restrict__ at0, const int *__restrict__ excl, const double *__restrict__ r,
      const double *__restrict__ q, double *__restrict__ F, double *__restrict__ partial, const SogConsts sc)
{
    __shared__ double red[32];
    const int c = blockIdx.x;
    const DevSys &d = sys[mchunk_sys[c]];
    const double L[3] = {d.L[0], d.L[1], d.L[2]};
    double ue = 0.0, ub = 0.0, ua = 0.0, wx[6] = {0, 0, 0, 0, 0, 0}, wb[6] = {0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < mchunk_n[c]; k += blockDim.x) {
        const int m = mchunk_m0[c] + k;
        // bonds
        for (int e = b_start[m]; e < b_start[m + 1]; ++e) {
            const int i = bonds[2 * e], j = bonds[2 * e + 1];
            double dv[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
            min_image(dv, L);
            double rr = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
            double dr = rr - br0[e];
            ub += bk[e] * dr * dr;
            double cf = -2.0 * bk[e] * dr / rr;
            double f[3] = {cf * dv[0], cf * dv[1], cf * dv[2]};
            for (int a = 0; a < 3; ++a) { F[3 * i + a] += f[a]; F[3 * j + a] -= f[a]; }
            wb[0] += f[0] * dv[0]; wb[1] += f[1] * dv[1]; wb[2] += f[2] * dv[2];
            wb[3] += f[0] * dv[1]; wb[4] += f[0] * dv[2]; wb[5] += f[1] * dv[2];
        }
        // angles (i, j centre, k)
        for (int e = a_start[m]; e < a_start[m + 1]; ++e) {
            const int i = angles[3 * e], j = angles[3 * e + 1], kk = angles[3 * e + 2];
            double d1[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
            double d2[3] = {r[3 * kk] - r[3 * j], r[3 * kk + 1] - r[3 * j + 1], r[3 * kk + 2] - r[3 * j + 2]};
            min_image(d1, L);
            min_image(d2, L);
            double r1 = sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
            double r2 = sqrt(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
            double cs = (d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2]) / (r1 * r2);
            cs = fmin(1.0, fmax(-1.0, cs));
            double th = acos(cs), sn = fmax(sqrt(1.0 - cs * cs), 1e-12);
            double dth = th - at0[e];
            ua += ak[e] * dth * dth;
            double g = 2.0 * ak[e] * dth / sn;
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
        // exclusion corrections
        for (int e = e_start[m]; e < e_start[m + 1]; ++e) {
            const int i = excl[2 * e], j = excl[2 * e + 1];
            double dv[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
            min_image(dv, L);
            double r2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
            double fe, ft;
            if (F32) {
                float r2f = (float)r2, a = 0.f, bsum = 0.f;
                for (int l = 0; l < sc.M; ++l) {
                    float ex = __expf(-r2f / (float)(sc.st[l] * sc.st[l]));
                    a = fmaf((float)sc.wt[l], ex, a);
                    bsum = fmaf((float)sc.w[l], ex, bsum);
                }
                for (int l = sc.M; l < sc.ME; ++l)
                    bsum = fmaf((float)sc.w[l], __expf(-r2f / (float)(sc.s[l] * sc.s[l])), bsum);
                ft = a;
                fe = bsum;
            } else {
                ft = 0.0; fe = 0.0;
                for (int l = 0; l < sc.M; ++l) {
                    double ex = exp(-r2 / (sc.st[l] * sc.st[l]));
                    ft += sc.wt[l] * ex;
                    fe += sc.w[l] * ex;
                }
                for (int l = sc.M; l < sc.ME; ++l) fe += sc.w[l] * exp(-r2 / (sc.s[l] * sc.s[l]));
            }
            double qq = sc.ke * q[i] * q[j];
            ue -= qq * fe;
            double f[3] = {-qq * ft * dv[0], -qq * ft * dv[1], -qq * ft * dv[2]};
            for (int a = 0; a < 3; ++a) { F[3 * i + a] += f[a]; F[3 * j + a] -= f[a]; }
            wx[0] += f[0] * dv[0]; wx[1] += f[1] * dv[1]; wx[2] += f[2] * dv[2];
            wx[3] += f[0] * dv[1]; wx[4] += f[0] * dv[2]; wx[5] += f[1] * dv[2];
        }
    }
    double v[15] = {ue, ub, ua, wx[0], wx[1], wx[2], wx[3], wx[4], wx[5],
                    wb[0], wb[1], wb[2], wb[3], wb[4], wb[5]};
    for (int k = 0; k < 15; ++k) {
        double t = block_sum(v[k], red);
        if (threadIdx.x == 0) partial[(size_t)c * 15 + k] = t;
    }
}

void launch_mol(const Batch &b, const AtomArrays &a, const MolArrays &m, const SogConsts &sc,
                double *partial, int precision, cudaStream_t st)
{
    if (m.nmchunks == 0) return;
    if (precision == 1)
        k_mol<true><<<m.nmchunks, 128, 0, st>>>(b.sys, m.mchunk_sys, m.mchunk_m0, m.mchunk_n, m.b_start,
                                               m.a_start, m.e_start, m.bonds, m.bk, m.br0, m.angles, m.ak,
                                               m.at0, m.excl, a.r, a.q, a.F, partial, sc);
    else
        k_mol<false><<<m.nmchunks, 128, 0, st>>>(b.sys, m.mchunk_sys, m.mchunk_m0, m.mchunk_n, m.b_start,
                                                m.a_start, m.e_start, m.bonds, m.bk, m.br0, m.angles, m.ak,
                                                m.at0, m.excl, a.r, a.q, a.F, partial, sc);
}

}  // namespace rbsog
