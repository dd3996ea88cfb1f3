// k_kspace.cu -- random-batch Fourier part (paper sec. 3.2, App. B).
//
//   rho(k_d) = sum_j q_j e^{i k_d . r_j} = sum_j q_j e^{2 pi i m_d . s_j}   (eq. rho_k)
//   U^F*     = ke S^r /(4 V P) sum_d c_r |rho_d|^2 / k_d^2                  (App. A with App. B's proposal)
//   V P^F,r* = ke S^r /(4 V P) sum_d c_r |rho_d|^2 / k_d^2 I                (eq. P_approx_r)
//   V P^F,nr*= -ke S^nr/(8 V P) sum_d c_nr |rho_d|^2 k_d (x) k_d / k_d^4   (eq. P_approx_nr)
//   F_i     += q_i sum_d alpha_d k_d Im(e^{-i k_d . r_i} rho_d),
//              alpha_d = -ke (S^r / 2) c_r / (P V k_d^2)                   (eq. f_approx)
// with the force proposal of App. B equal to P^r and its normaliser S = S^r/2
// for the consistent split (w_l = w~_l s~_l^2 / 2, App. C).
//
// FP32 build: the phase m.s mod 1 is formed exactly in 32-bit integer
// arithmetic on fixed-point fractional coordinates (s 2^32), then its sine
// and cosine from a 256-entry table and the remainder's short Taylor forms
// (phase_sincos_f); per-lane sums are compensated FP32, lane/chunk sums FP64.  FP64 build: phases and sums in FP64.
#include "internal.h"

namespace rbsog {

namespace {

constexpr int kModeGroup = 16;   // modes per block of the S(k) kernel
constexpr int kSkThreads = 256;  // 8 warps: one or two modes each
constexpr int kSkSmallGrid = 152;   // this GPU's SM count: an FP64 S(k) grid below it halves its mode groups

struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Table of (cos, sin)(2 pi k / 256), k < 256, for phase_sincos_f; filled by
// the threads of a block (sincospif of exact arguments k / 128), which must
// synchronise before the first use.
constexpr int kTurnTab = 256;
__device__ __forceinline__ void fill_turn_table(float2 *tab)
{
    for (int k = threadIdx.x; k < kTurnTab; k += blockDim.x) {
        float sn, cs;
        sincospif((float)k * (1.0f / 128.0f), &sn, &cs);
        tab[k] = make_float2(cs, sn);
    }
}

// sin and cos of 2 pi (m . s) for fixed-point fractional coordinates s 2^32:
// the phase ph = m . s 2^32 mod 2^32 is exact in 32-bit integer arithmetic;
// ph = 2^24 k + r with k the nearest of 256 table angles and |r| <= 2^23, so
// the remainder angle b = 2 pi r / 2^32 has |b| <= pi / 256, where sin b =
// b - b^3/6 (next term below 2.4e-12) and cos b = 1 - b^2/2 (next term below
// 9.4e-10) are exact to FP32 rounding; the angle-sum formulas combine them
// with the table (about as accurate as sincospif, in a third of the
// instructions).
__device__ __forceinline__ void phase_sincos_f(const int m[3], uint4 su, const float2 *tab, float &sn, float &cs)
{
    const unsigned ph = (unsigned)m[0] * su.x + (unsigned)m[1] * su.y + (unsigned)m[2] * su.z;
    const unsigned k = (ph + 0x800000u) >> 24;
    const float b = (float)(int)(ph - (k << 24)) * 1.4629180792671596e-09f;   // 2 pi / 2^32
    const float b2 = b * b;
    const float sb = fmaf(b * b2, -0.16666667f, b);
    const float cb = fmaf(b2, -0.5f, 1.0f);
    const float2 t = tab[k & (kTurnTab - 1)];
    sn = fmaf(t.y, cb, t.x * sb);
    cs = fmaf(t.x, cb, -(t.y * sb));
}

__device__ __forceinline__ void phase_sincos_d(const int m[3], double sx, double sy, double sz,
                                               double &sn, double &cs)
{
    double t = (double)m[0] * sx + (double)m[1] * sy + (double)m[2] * sz;
    t -= rint(t);
    sincospi(2.0 * t, &sn, &cs);
}

// FP64 table of (cos, sin)(2 pi k / 512), k < 512, for phase_sincos_dt;
// filled by the threads of a block (sincospi of exact arguments k / 256),
// which must synchronise before the first use.
constexpr int kTurnTabD = 512;
static_assert(kTurnTabD == kTurnTabEntries, "the context allocates kTurnTabEntries table entries");
__device__ __forceinline__ void fill_turn_table_d(double2 *tab)
{
    for (int k = threadIdx.x; k < kTurnTabD; k += blockDim.x) {
        double sn, cs;
        sincospi((double)k * (1.0 / 256.0), &sn, &cs);
        tab[k] = make_double2(cs, sn);
    }
}

// The FP64 table in shared memory: copied from gtab (the context's copy, made
// once by k_turn_table_d with the same function) or, without one, filled here.
__device__ __forceinline__ void load_turn_table_d(double2 *tab, const double2 *__restrict__ gtab)
{
    if (gtab)
        for (int k = threadIdx.x; k < kTurnTabD; k += blockDim.x) tab[k] = gtab[k];
    else
        fill_turn_table_d(tab);
}

// sin and cos of 2 pi (m . s) in FP64 from the table: t = m . s mod 1 as in
// phase_sincos_d, 512 t = k + b with k the nearest integer (|b| <= 1/2, exact),
// the remainder angle c = 2 pi b / 512 has |c| <= pi / 512, where
// sin c = c (1 - c^2/6 + c^4/120) (next term below 1e-19 of c) and
// cos c = 1 - c^2/2 + c^4/24 - c^6/720 (next term below 3e-21); the
// angle-sum formulas combine them with the table: about half the FP64
// instructions of sincospi, and as accurate.
__device__ __forceinline__ void phase_sincos_dt(const int m[3], double sx, double sy, double sz,
                                                const double2 *tab, double &sn, double &cs)
{
    double t = (double)m[0] * sx + (double)m[1] * sy + (double)m[2] * sz;
    t -= rint(t);
    const double u = t * (double)kTurnTabD;
    const double kf = rint(u);
    const double c = (u - kf) * (kTwoPi / (double)kTurnTabD);
    const double c2 = c * c;
    const double sc = c * fma(c2, fma(c2, 1.0 / 120.0, -1.0 / 6.0), 1.0);
    const double cc = fma(c2, fma(c2, fma(c2, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
    const double2 tb = tab[(int)kf & (kTurnTabD - 1)];
    sn = fma(tb.y, cc, tb.x * sc);
    cs = fma(tb.x, cc, -(tb.y * sc));
}

// rho partial sums of one chunk of atoms for a group of modes.
// su: FP32 atom data (fixed-point s, q bits); r/q/L: FP64 atom data.
// B: the edges L and, for a tilted cell, the tilts (xy, xz, yz) in B[3..5]
// (null: orthorhombic); the FP64 phases use s = h^{-1} r.
template <bool F32>
__device__ void sk_chunk(const uint4 *su, const double *r, const double *q, const double L[3], const double *tilt,
                         int a0, int na, const int *D, int d0, int nd_here, double *out /* [nd_here][2] */,
                         const double2 *gtab = nullptr)
{
    __shared__ uint4 s_su[F32 ? kChunk : 1];
    __shared__ double s_sd[F32 ? 1 : kChunk][4];
    __shared__ float2 s_tab[F32 ? kTurnTab : 1];
    __shared__ double2 s_tabd[F32 ? 1 : kTurnTabD];
    if (F32) fill_turn_table(s_tab);
    else load_turn_table_d(s_tabd, gtab);
    const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5, nw = blockDim.x >> 5;
    for (int k = tid; k < na; k += blockDim.x) {
        if (F32) {
            s_su[k] = su[a0 + k];
        } else {
            const int i = a0 + k;
            if (tilt) {
                const double sz = r[3 * i + 2] / L[2];
                const double sy = (r[3 * i + 1] - tilt[2] * sz) / L[1];
                s_sd[k][0] = (r[3 * i] - tilt[0] * sy - tilt[1] * sz) / L[0];
                s_sd[k][1] = sy;
                s_sd[k][2] = sz;
            } else {
                s_sd[k][0] = r[3 * i] / L[0];
                s_sd[k][1] = r[3 * i + 1] / L[1];
                s_sd[k][2] = r[3 * i + 2] / L[2];
            }
            s_sd[k][3] = q[i];
        }
    }
    __syncthreads();
    for (int dd = warp; dd < nd_here; dd += nw) {
        const int m[3] = {D[3 * (d0 + dd)], D[3 * (d0 + dd) + 1], D[3 * (d0 + dd) + 2]};
        double re, im;
        if (F32) {
            Kahan kr, ki;
            for (int k = lane; k < na; k += 32) {
                uint4 v = s_su[k];
                float sn, cs;
                phase_sincos_f(m, v, s_tab, sn, cs);
                float qq = __uint_as_float(v.w);
                kr.add(qq * cs);
                ki.add(qq * sn);
            }
            re = warp_sum(kr.value());
            im = warp_sum(ki.value());
        } else {
            double sr = 0.0, si = 0.0;
            for (int k = lane; k < na; k += 32) {
                double sn, cs;
                phase_sincos_dt(m, s_sd[k][0], s_sd[k][1], s_sd[k][2], s_tabd, sn, cs);
                sr += s_sd[k][3] * cs;
                si += s_sd[k][3] * sn;
            }
            re = warp_sum(sr);
            im = warp_sum(si);
        }
        if (lane == 0) {
            out[2 * dd] = re;
            out[2 * dd + 1] = im;
        }
    }
}

}  // namespace

// grid: (nchunks x nsub, ceil(Dcap / kModeGroup)), nsub = 1 (FP32) or kSkSubD
// (FP64) sub-chunks of kChunk / nsub atoms; part[chunk][sub][Dcap][2]
template <bool F32>
__global__ void __launch_bounds__(kSkThreads)
k_sk(const DevSys *__restrict__ sys, const int *__restrict__ chunk_sys, const int *__restrict__ chunk_a0,
     const int *__restrict__ chunk_n, const uint4 *__restrict__ su, const double *__restrict__ r,
     const double *__restrict__ q, const int *__restrict__ D, int Dcap, double *__restrict__ part,
     const double2 *__restrict__ gtab, int mg)
{
    constexpr int nsub = F32 ? 1 : kSkSubD, span = kChunk / nsub;
    const int c = blockIdx.x / nsub, sb = blockIdx.x % nsub, s = chunk_sys[c];
    const DevSys &d = sys[s];
    const int d0 = blockIdx.y * mg;
    // atoms of this sub-chunk (<= 0: beyond the system in its slot)
    const int na = min(span, live_n(d) - (chunk_a0[c] - d.atom0) - sb * span);
    if (d0 >= d.nD || na <= 0) return;
    const int nd_here = min(mg, d.nD - d0);
    const double L[3] = {d.L[0], d.L[1], d.L[2]};
    sk_chunk<F32>(su, r, q, L, d.tri ? d.tilt : nullptr, chunk_a0[c] + sb * span, na, D + (size_t)s * Dcap * 3, d0,
                  nd_here, part + ((size_t)blockIdx.x * Dcap + d0) * 2, gtab);
}

void launch_sk(const Batch &b, const AtomArrays &a, int precision, const int *D, int Dcap,
               double *part, cudaStream_t st)
{
    // modes per block: kModeGroup, or half of it for an FP64 batch whose grid
    // would fill fewer blocks than the GPU has SMs (one warp per mode then);
    // each mode's sum runs over the same atoms in the same order either way
    const int nx = b.nchunks * sk_sub(precision);
    const int mg = (precision != 1 && nx * ((Dcap + kModeGroup - 1) / kModeGroup) < kSkSmallGrid) ? kModeGroup / 2
                                                                                                   : kModeGroup;
    dim3 grid(nx, (Dcap + mg - 1) / mg);
    if (precision == 1)
        k_sk<true><<<grid, kSkThreads, 0, st>>>(b.sys, b.chunk_sys, b.chunk_a0, b.chunk_n, a.su, a.r, a.q,
                                               D, Dcap, part, nullptr, mg);
    else
        k_sk<false><<<grid, kSkThreads, 0, st>>>(b.sys, b.chunk_sys, b.chunk_a0, b.chunk_n, a.su, a.r, a.q,
                                                D, Dcap, part, a.turn_tab_d, mg);
}

__global__ void k_turn_table_d(double2 *tab) { fill_turn_table_d(tab); }

void launch_turn_table_d(double2 *tab, cudaStream_t st) { k_turn_table_d<<<1, kTurnTabD, 0, st>>>(tab); }

// One block per (system, group of 32 modes).  Warp w sums its share of the
// chunk partials of rho (fixed chunk ranges, in chunk order), warp 0 adds the
// shares in warp order and computes, per mode, the force coefficients and the
// mode's terms of the estimators; the group's sums go to
// est[(s * groups + g) * 7 + t] = {sum c_r |rho|^2 / k^2,
// sum c_nr |rho|^2 k (x) k / k^4 (xx yy zz xy xz yz)}, and k_finalize adds the
// groups in order and applies the prefactors (eqs. U_F*, P_F,r*, P_F,nr*).
constexpr int kEstModes = 32, kEstWarps = 4;

int estimate_blocks(int Dcap) { return (Dcap + kEstModes - 1) / kEstModes; }

__global__ void __launch_bounds__(32 * kEstWarps)
k_estimate(const DevSys *sys, const int *__restrict__ first_chunk, const int *__restrict__ nchunk_sys,
           const int *__restrict__ D_all, const int *__restrict__ cr_all, const int *__restrict__ cnr_all,
           int Dcap, int P, double ke, const double *__restrict__ part, double *__restrict__ rho_all,
           ModeCoef *__restrict__ coef_all, double *__restrict__ est, int nsub)
{
    __shared__ double2 sh[kEstWarps][kEstModes];
    const int s = blockIdx.x, g = blockIdx.y, w = threadIdx.x >> 5, lane = lane_id();
    const DevSys &d = sys[s];
    const int nD = d.nD, k = g * kEstModes + lane;
    // (sub-)chunks holding atoms of the system (its slot may have more), in order
    const int span = kChunk / nsub;
    const int c0 = first_chunk[s] * nsub, nc = min(nchunk_sys[s] * nsub, (live_n(d) + span - 1) / span);
    const int cb = (int)((long long)nc * w / kEstWarps), ce = (int)((long long)nc * (w + 1) / kEstWarps);
    double re = 0.0, im = 0.0;
    if (k < nD) {
        const double2 *pk = reinterpret_cast<const double2 *>(part) + (size_t)c0 * Dcap + k;
        int c = cb;
        for (; c + 4 <= ce; c += 4) {          // loads issued together, sums in chunk order
            double2 t[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) t[u] = pk[(size_t)(c + u) * Dcap];
#pragma unroll
            for (int u = 0; u < 4; ++u) { re += t[u].x; im += t[u].y; }
        }
        for (; c < ce; ++c) { const double2 t = pk[(size_t)c * Dcap]; re += t.x; im += t.y; }
    }
    sh[w][lane] = make_double2(re, im);
    __syncthreads();
    if (w != 0) return;
    double il = 0.0;                           // lane a < 3: 1 / L_a
    if (lane < 3) il = 1.0 / d.L[lane];
    const double ilx = __shfl_sync(0xffffffffu, il, 0), ily = __shfl_sync(0xffffffffu, il, 1),
                 ilz = __shfl_sync(0xffffffffu, il, 2);
    const double iV = ilx * ily * ilz;
    double v[7] = {0, 0, 0, 0, 0, 0, 0};
    if (k < nD) {
        re = sh[0][lane].x;
        im = sh[0][lane].y;
#pragma unroll
        for (int u = 1; u < kEstWarps; ++u) { re += sh[u][lane].x; im += sh[u][lane].y; }
        double *rho = rho_all + (size_t)s * Dcap * 2;
        rho[2 * k] = re;
        rho[2 * k + 1] = im;
        const int *D = D_all + ((size_t)s * Dcap + k) * 3;
        const int m0 = D[0], m1 = D[1], m2 = D[2];
        double kx = kTwoPi * m0 * ilx, ky = kTwoPi * m1 * ily, kz = kTwoPi * m2 * ilz;
        if (d.tri) {                           // k = 2 pi h^{-T} m
            const int mm[3] = {m0, m1, m2};
            double kk[3];
            kvec_of(d, mm, kk);
            kx = kk[0]; ky = kk[1]; kz = kk[2];
        }
        const double ik2 = 1.0 / (kx * kx + ky * ky + kz * kz);
        const double r2 = re * re + im * im;
        const double cr = cr_all[(size_t)s * Dcap + k], cnr = cnr_all[(size_t)s * Dcap + k];
        v[0] = cr * r2 * ik2;
        const double gg = cnr * r2 * ik2 * ik2;
        v[1] = gg * kx * kx; v[2] = gg * ky * ky; v[3] = gg * kz * kz;
        v[4] = gg * kx * ky; v[5] = gg * kx * kz; v[6] = gg * ky * kz;
        const double alpha = -ke * (0.5 * d.Sr) / P * iV * cr * ik2;
        ModeCoef mc;
        mc.a[0] = alpha * kx; mc.a[1] = alpha * ky; mc.a[2] = alpha * kz;
        mc.re = re; mc.im = im;
        mc.m[0] = m0; mc.m[1] = m1; mc.m[2] = m2;
        mc.pad = 0;
        coef_all[(size_t)s * Dcap + k] = mc;
    }
#pragma unroll
    for (int t = 0; t < 7; ++t) v[t] = warp_sum(v[t]);
    if (lane < 7) {
        double x = v[0];
#pragma unroll
        for (int t = 1; t < 7; ++t)
            if (lane == t) x = v[t];
        est[((size_t)s * gridDim.y + g) * 7 + lane] = x;
    }
}

void launch_estimate(const Batch &b, const int *first_chunk, const int *nchunk_sys, const int *D,
                     const int *cr, const int *cnr, int Dcap, int P, double ke, const double *part,
                     double *rho, ModeCoef *coef, double *est, cudaStream_t st, int precision)
{
    k_estimate<<<dim3(b.S, estimate_blocks(Dcap)), 32 * kEstWarps, 0, st>>>(
        b.sys, first_chunk, nchunk_sys, D, cr, cnr, Dcap, P, ke, part, rho, coef, est, sk_sub(precision));
}

// Long-range force (eq. f_approx): F^lr_i = q_i sum_d alpha_d k_d
// Im(e^{-i k_d.r_i} rho_d), written per atom to Flr.  It needs the modes'
// coefficients and the atoms' positions only, so in the FP32 build it runs on
// the sampler's stream beside the pair kernel.  Blocks of kLrAtoms atoms of
// one chunk and one group of modes (grid: chunks x kChunk / kLrAtoms x
// lr_groups; the FP64 build's kLrGroupsD groups each write a partial force
// Flr + g 3N); the group's mode coefficients are staged in shared memory in
// tiles.
constexpr int kModeTile = 256;
constexpr int kLrAtoms = kChunk / kKinSplit;

template <bool F32>
__global__ void __launch_bounds__(kLrAtoms)
k_lr_fourier(const DevSys *__restrict__ sys, const int *__restrict__ chunk_sys, const int *__restrict__ chunk_a0,
             const uint4 *__restrict__ su, const double *__restrict__ r, const double *__restrict__ q,
             const ModeCoef *__restrict__ coef_all, int Dcap, double *__restrict__ Flr, int N,
             const double2 *__restrict__ gtab)
{
    __shared__ float4 tf[F32 ? kModeTile : 1];      // a (FP32)
    __shared__ float2 tr[F32 ? kModeTile : 1];      // re, im
    __shared__ int4 tm[kModeTile];
    __shared__ double td[F32 ? 1 : kModeTile][5];
    __shared__ float2 tab[F32 ? kTurnTab : 1];
    __shared__ double2 tabd[F32 ? 1 : kTurnTabD];
    const int c = blockIdx.x, s = chunk_sys[c];
    const DevSys &d = sys[s];
    const int nD = d.nD, a0 = chunk_a0[c], na = min(kChunk, live_n(d) - (a0 - d.atom0));
    const ModeCoef *coef = coef_all + (size_t)s * Dcap;
    const int k = blockIdx.y * kLrAtoms + threadIdx.x;
    if ((int)(blockIdx.y * kLrAtoms) >= na) return;   // whole block beyond the chunk
    // this block's modes: group blockIdx.z of lr_groups (FP32: all of them);
    // a group without modes writes zeros
    constexpr int G = F32 ? 1 : kLrGroupsD;
    const int per = (nD + G - 1) / G;
    const int mb = min(nD, (int)blockIdx.z * per), me = min(nD, mb + per);
    Flr += (size_t)blockIdx.z * 3 * N;
    if (F32) fill_turn_table(tab);                    // used after the tile loop's barrier
    else load_turn_table_d(tabd, gtab);
    const bool act = k < na;
    const int i = a0 + (act ? k : 0);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    double gx = 0.0, gy = 0.0, gz = 0.0;
    uint4 v = make_uint4(0, 0, 0, 0);
    double sx = 0.0, sy = 0.0, sz = 0.0;
    if (F32) v = su[i];
    else if (d.tri) {
        const double x[3] = {r[3 * i], r[3 * i + 1], r[3 * i + 2]};
        double sf[3];
        frac_of(d, x, sf);
        sx = sf[0]; sy = sf[1]; sz = sf[2];
    } else { sx = r[3 * i] / d.L[0]; sy = r[3 * i + 1] / d.L[1]; sz = r[3 * i + 2] / d.L[2]; }
    for (int t0 = mb; t0 < me; t0 += kModeTile) {
        const int nt = min(kModeTile, me - t0);
        __syncthreads();
        for (int u = threadIdx.x; u < nt; u += blockDim.x) {
            const ModeCoef &mc = coef[t0 + u];
            if (F32) {
                tf[u] = make_float4((float)mc.a[0], (float)mc.a[1], (float)mc.a[2], 0.f);
                tr[u] = make_float2((float)mc.re, (float)mc.im);
            } else {
                td[u][0] = mc.a[0]; td[u][1] = mc.a[1]; td[u][2] = mc.a[2];
                td[u][3] = mc.re; td[u][4] = mc.im;
            }
            tm[u] = make_int4(mc.m[0], mc.m[1], mc.m[2], 0);
        }
        __syncthreads();
        if (F32) {
#pragma unroll 4
            for (int u = 0; u < nt; ++u) {
                const int4 mm = tm[u];
                const int m[3] = {mm.x, mm.y, mm.z};
                const float4 av = tf[u];
                const float2 rr = tr[u];
                float sn, cs;
                phase_sincos_f(m, v, tab, sn, cs);
                const float g = rr.y * cs - rr.x * sn;
                fx = fmaf(av.x, g, fx);
                fy = fmaf(av.y, g, fy);
                fz = fmaf(av.z, g, fz);
            }
        } else {
            for (int u = 0; u < nt; ++u) {
                const int4 mm = tm[u];
                const int m[3] = {mm.x, mm.y, mm.z};
                double sn, cs;
                phase_sincos_dt(m, sx, sy, sz, tabd, sn, cs);
                const double g = td[u][4] * cs - td[u][3] * sn;
                gx += td[u][0] * g;
                gy += td[u][1] * g;
                gz += td[u][2] * g;
            }
        }
    }
    if (act) {
        const double qi = q[i];
        if (F32) {
            Flr[3 * i] = qi * (double)fx;
            Flr[3 * i + 1] = qi * (double)fy;
            Flr[3 * i + 2] = qi * (double)fz;
        } else {
            Flr[3 * i] = qi * gx;
            Flr[3 * i + 1] = qi * gy;
            Flr[3 * i + 2] = qi * gz;
        }
    }
}

void launch_lr_fourier(const Batch &b, const AtomArrays &a, int precision, const ModeCoef *coef, int Dcap,
                       double *Flr, cudaStream_t st)
{
    const dim3 grid(b.nchunks, kChunk / kLrAtoms, lr_groups(precision));
    if (precision == 1)
        k_lr_fourier<true><<<grid, kLrAtoms, 0, st>>>(b.sys, b.chunk_sys, b.chunk_a0, a.su, a.r, a.q, coef, Dcap, Flr,
                                                     b.N, nullptr);
    else
        k_lr_fourier<false><<<grid, kLrAtoms, 0, st>>>(b.sys, b.chunk_sys, b.chunk_a0, a.su, a.r, a.q, coef, Dcap, Flr,
                                                      b.N, a.turn_tab_d);
}

// Force assembly: F_i = the pair kernel's fixed-point sum (read and cleared)
// + the long-range force Flr (k_lr_fourier, its mode groups in order) + the
// molecule terms of k_mol, in that order.  The same blocks (kLrAtoms atoms of one chunk) then give the
// atoms their second half kick (velocity Verlet B step) and sum the kinetic
// tensor p (x) p / m of their atoms, one partial per block.
template <bool F32>
__global__ void __launch_bounds__(kLrAtoms)
k_force_assembly(const DevSys *__restrict__ sys, const int *__restrict__ chunk_sys, const int *__restrict__ chunk_a0,
                 const double *__restrict__ Flr, const int *__restrict__ pos_sorted,
                 unsigned long long *__restrict__ ffix, int N, const double *__restrict__ Fmol,
                 double *__restrict__ F, double *__restrict__ mom, const double *__restrict__ inv_m, double kick,
                 double mvv2e, double *__restrict__ kin_part)
{
    __shared__ double red[6 * (kLrAtoms + 1) + 24];
    const int c = blockIdx.x, s = chunk_sys[c];
    const DevSys &d = sys[s];
    const int a0 = chunk_a0[c], na = min(kChunk, live_n(d) - (a0 - d.atom0));
    const int k = blockIdx.y * kLrAtoms + threadIdx.x;
    double *kin = kin_part + ((size_t)c * kKinSplit + blockIdx.y) * 6;
    if ((int)(blockIdx.y * kLrAtoms) >= na) {         // whole block beyond the chunk
        if (threadIdx.x < 6) kin[threadIdx.x] = 0.0;
        return;
    }
    const bool act = k < na;
    const int i = a0 + (act ? k : 0);
    double k6[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (act) {
        const int ks = pos_sorted[i];
        double f[3] = {0.0, 0.0, 0.0};
        // fixed-point pair forces (FP64: two words), cleared for the next evaluation
        if (F32) {
            for (int a = 0; a < 3; ++a) {
                f[a] = (double)(long long)ffix[(size_t)a * N + ks] * (1.0 / kFixScale);
                ffix[(size_t)a * N + ks] = 0ull;
            }
        } else {
            for (int a = 0; a < 3; ++a) {
                const long long h = (long long)ffix[(size_t)a * N + ks], l = (long long)ffix[(size_t)(3 + a) * N + ks];
                f[a] = (double)h * (1.0 / kFix2Scale) + (double)l * (1.0 / (kFix2Scale * kFix2Scale));
                ffix[(size_t)a * N + ks] = 0ull;
                ffix[(size_t)(3 + a) * N + ks] = 0ull;
            }
        }
        constexpr int G = F32 ? 1 : kLrGroupsD;     // the long-range force's mode groups, in order
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const double *fl = Flr + (size_t)g * 3 * N;
            f[0] += fl[3 * i];
            f[1] += fl[3 * i + 1];
            f[2] += fl[3 * i + 2];
        }
        if (Fmol) {
            f[0] += Fmol[3 * i];
            f[1] += Fmol[3 * i + 1];
            f[2] += Fmol[3 * i + 2];
        }
        F[3 * i] = f[0];
        F[3 * i + 1] = f[1];
        F[3 * i + 2] = f[2];
        double v[3];
        for (int a = 0; a < 3; ++a) {
            v[a] = mom[3 * i + a];
            if (kick != 0.0) {
                v[a] += kick * f[a];
                mom[3 * i + a] = v[a];
            }
        }
        const double im = inv_m[i];
        k6[0] = v[0] * v[0] * im * mvv2e; k6[1] = v[1] * v[1] * im * mvv2e; k6[2] = v[2] * v[2] * im * mvv2e;
        k6[3] = v[0] * v[1] * im * mvv2e; k6[4] = v[0] * v[2] * im * mvv2e; k6[5] = v[1] * v[2] * im * mvv2e;
    }
    block_reduce_lanes<6, kLrAtoms>(k6, red, kin);
}

void launch_force_assembly(const Batch &b, const AtomArrays &a, int precision, const double *Flr,
                           const double *Fmol, const IntegArgs &ia, int do_kick, double *kin_part, cudaStream_t st)
{
    const double kick = do_kick ? 0.5 * ia.dt * ia.ftm2v : 0.0, mvv2e = 1.0 / ia.ftm2v;
    const dim3 grid(b.nchunks, kChunk / kLrAtoms);
    if (precision == 1)
        k_force_assembly<true><<<grid, kLrAtoms, 0, st>>>(b.sys, b.chunk_sys, b.chunk_a0, Flr, a.rank, a.ffix, b.N,
                                                          Fmol, a.F, a.p, ia.inv_m, kick, mvv2e, kin_part);
    else
        k_force_assembly<false><<<grid, kLrAtoms, 0, st>>>(b.sys, b.chunk_sys, b.chunk_a0, Flr, a.rank, a.ffix, b.N,
                                                           Fmol, a.F, a.p, ia.inv_m, kick, mvv2e, kin_part);
}

// Shared-proposal estimator of the non-radial virial (sec. 3.2, the
// alternative the measure recalibration replaces): the radial samples reused
// for P^F,nr with weights f_nr / P^r = S^r k^2 R(k), R(k) = sum_l cn_l e_l /
// sum_l cr_l e_l, e_l = e^{-s~_l^2 k^2 / 4} (eqs. samplingP, samplingPnr):
//   V P^F,nr,sh = -ke S^r / (8 V P) sum_d c_r[d] R(k_d) |rho_d|^2 k (x) k / k^2
// over the modes and structure factors of the last evaluation.  One block per
// system; used to compare estimators, not part of the MD step.
constexpr int kNrShThreads = 128;

__global__ void __launch_bounds__(kNrShThreads)
k_nr_shared(const DevSys *__restrict__ sys, const int *__restrict__ D_all, const int *__restrict__ cr_all,
            const double *__restrict__ rho_all, int Dcap, int P, double ke, const SamplerArgs sa,
            double *__restrict__ out)
{
    __shared__ double red[6 * (kNrShThreads + 1) + 24];
    __shared__ double tot[6];
    const int s = blockIdx.x;
    const DevSys &d = sys[s];
    const int nD = live_n(d) > 0 ? d.nD : 0;
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < nD; k += blockDim.x) {
        const int *Dk = D_all + ((size_t)s * Dcap + k) * 3;
        double kx = kTwoPi * Dk[0] / d.L[0], ky = kTwoPi * Dk[1] / d.L[1], kz = kTwoPi * Dk[2] / d.L[2];
        if (d.tri) {
            double kk[3];
            kvec_of(d, Dk, kk);
            kx = kk[0]; ky = kk[1]; kz = kk[2];
        }
        const double k2 = kx * kx + ky * ky + kz * kz;
        double a = 0.0, b = 0.0;
        for (int l = 0; l < sa.M; ++l) {
            const double e = exp(-(sa.st2q[l] * k2));
            a += sa.cr[l] * e;
            b += sa.cn[l] * e;
        }
        const double *rh = rho_all + ((size_t)s * Dcap + k) * 2;
        const double g = cr_all[(size_t)s * Dcap + k] * (b / a) * (rh[0] * rh[0] + rh[1] * rh[1]) / k2;
        v[0] += g * kx * kx; v[1] += g * ky * ky; v[2] += g * kz * kz;
        v[3] += g * kx * ky; v[4] += g * kx * kz; v[5] += g * ky * kz;
    }
    block_reduce_lanes<6, kNrShThreads>(v, red, tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double c = -ke * d.Sr / (8.0 * (d.L[0] * d.L[1] * d.L[2]) * P);
        double *o = out + (size_t)s * 9;
        o[0] = c * tot[0]; o[4] = c * tot[1]; o[8] = c * tot[2];
        o[1] = o[3] = c * tot[3];
        o[2] = o[6] = c * tot[4];
        o[5] = o[7] = c * tot[5];
    }
}

void launch_nr_shared(const Batch &b, const int *D, const int *cr, const double *rho, int Dcap, int P, double ke,
                      const SamplerArgs &sa, double *out, cudaStream_t st)
{
    k_nr_shared<<<b.S, kNrShThreads, 0, st>>>(b.sys, D, cr, rho, Dcap, P, ke, sa, out);
}

// ---------------------------------------------------------------------------
// stateless structure factor on caller buffers
// ---------------------------------------------------------------------------
__global__ void k_su_from_r(const double *__restrict__ r, const double *__restrict__ q, int n, double L0,
                            double L1, double L2, uint4 *__restrict__ su)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double L[3] = {L0, L1, L2};
    unsigned f[3];
    for (int a = 0; a < 3; ++a) {
        double s = r[3 * i + a] / L[a];
        s -= floor(s);
        if (s >= 1.0) s = 0.0;
        f[a] = __double2uint_rz(s * 4294967296.0);
    }
    su[i] = make_uint4(f[0], f[1], f[2], __float_as_uint((float)q[i]));
}

template <bool F32>
__global__ void __launch_bounds__(kSkThreads)
k_sk_stateless(const uint4 *__restrict__ su, const double *__restrict__ r, const double *__restrict__ q,
               int n, double L0, double L1, double L2, const int *__restrict__ m, int nD,
               double *__restrict__ part)
{
    const int c = blockIdx.x, d0 = blockIdx.y * kModeGroup;
    if (d0 >= nD) return;
    const int a0 = c * kChunk, na = min(kChunk, n - a0);
    const double L[3] = {L0, L1, L2};
    sk_chunk<F32>(su, r, q, L, nullptr, a0, na, m, d0, min(kModeGroup, nD - d0), part + ((size_t)c * nD + d0) * 2);
}

__global__ void k_sk_reduce(const double *__restrict__ part, int nchunks, int nD, double *__restrict__ rho)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * nD) return;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += part[(size_t)c * nD * 2 + k];
    rho[k] = s;
}

size_t sk_stateless_workspace(int n, int nD)
{
    const size_t nch = (size_t)(n + kChunk - 1) / kChunk;
    size_t part = nch * (size_t)nD * 2 * sizeof(double);
    size_t su = (size_t)n * sizeof(uint4);
    return ((part + 255) / 256) * 256 + su;
}

cudaError_t sk_stateless(const double *r, const double *q, int n, const double box[3], const int *m, int nD,
                         double *rho, void *work, int precision, cudaStream_t st)
{
    const int nch = (n + kChunk - 1) / kChunk;
    double *part = static_cast<double *>(work);
    size_t part_b = ((nch * (size_t)nD * 2 * sizeof(double) + 255) / 256) * 256;
    uint4 *su = reinterpret_cast<uint4 *>(static_cast<char *>(work) + part_b);
    dim3 grid(nch, (nD + kModeGroup - 1) / kModeGroup);
    if (precision == 1) {
        k_su_from_r<<<(n + 255) / 256, 256, 0, st>>>(r, q, n, box[0], box[1], box[2], su);
        k_sk_stateless<true><<<grid, kSkThreads, 0, st>>>(su, r, q, n, box[0], box[1], box[2], m, nD, part);
    } else {
        k_sk_stateless<false><<<grid, kSkThreads, 0, st>>>(su, r, q, n, box[0], box[1], box[2], m, nD, part);
    }
    k_sk_reduce<<<(2 * nD + 255) / 256, 256, 0, st>>>(part, nch, nD, rho);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// stateless long-range force and estimators from given structure factors
// (the per-rank step of the single-system decomposition: rho summed over
// every rank's atoms, then each rank's own atoms)
// ---------------------------------------------------------------------------
constexpr int kLrsThreads = 128;

// per mode: alpha_d k_d (force coefficient, eq. f_approx) and the estimator
// terms; one thread per mode
__global__ void k_lrs_coef(const int *__restrict__ m, const int *__restrict__ cr, const int *__restrict__ cnr,
                           const double *__restrict__ rho, int nD, double L0, double L1, double L2, int P,
                           double Sr, double Snr, double ke, double4 *__restrict__ coef, double *__restrict__ terms)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= nD) return;
    const double V = L0 * L1 * L2;
    const double k[3] = {kTwoPi * m[3 * d] / L0, kTwoPi * m[3 * d + 1] / L1, kTwoPi * m[3 * d + 2] / L2};
    const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    const double a = -ke * 0.5 * Sr * (double)cr[d] / ((double)P * V * k2);
    coef[d] = make_double4(a * k[0], a * k[1], a * k[2], 0.0);
    const double r2 = rho[2 * d] * rho[2 * d] + rho[2 * d + 1] * rho[2 * d + 1];
    // U^F* (= tr V P^F,r* / 3) and V P^F,nr* (xx yy zz xy xz yz), summed over
    // the modes in order by k_lrs_sum
    const double ur = ke * Sr / (4.0 * V * P) * (double)cr[d] * r2 / k2;
    const double cn = cnr ? -ke * Snr / (8.0 * V * P) * (double)cnr[d] * r2 / (k2 * k2) : 0.0;
    double *t = terms + 7 * (size_t)d;
    t[0] = ur;
    t[1] = cn * k[0] * k[0]; t[2] = cn * k[1] * k[1]; t[3] = cn * k[2] * k[2];
    t[4] = cn * k[0] * k[1]; t[5] = cn * k[0] * k[2]; t[6] = cn * k[1] * k[2];
}

__global__ void k_lrs_sum(const double *__restrict__ terms, int nD, double *__restrict__ out)
{
    const int c = threadIdx.x;
    if (c >= 7) return;
    double s = 0.0;
    for (int d = 0; d < nD; ++d) s += terms[7 * (size_t)d + c];
    out[c] = s;
}

template <bool F32>
__global__ void __launch_bounds__(kLrsThreads)
k_lrs_force(const double *__restrict__ r, const double *__restrict__ q, int n, double L0, double L1, double L2,
            const int *__restrict__ m, const double *__restrict__ rho, const double4 *__restrict__ coef, int nD,
            double *__restrict__ F)
{
    __shared__ int4 tm[kModeTile];
    __shared__ double tc[kModeTile][5];
    __shared__ float2 ttab[F32 ? kTurnTab : 1];
    if (F32) fill_turn_table(ttab);                   // used after the tile loop's barrier
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = i < n;
    double sx = 0.0, sy = 0.0, sz = 0.0;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (act) {
        const double L[3] = {L0, L1, L2};
        double s3[3];
        unsigned f[3];
        for (int a = 0; a < 3; ++a) {
            double s = r[3 * i + a] / L[a];
            s -= floor(s);
            if (s >= 1.0) s = 0.0;
            s3[a] = s;
            f[a] = __double2uint_rz(s * 4294967296.0);
        }
        sx = s3[0]; sy = s3[1]; sz = s3[2];
        v = make_uint4(f[0], f[1], f[2], 0u);
    }
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int t0 = 0; t0 < nD; t0 += kModeTile) {
        const int nt = min(kModeTile, nD - t0);
        __syncthreads();
        for (int u = threadIdx.x; u < nt; u += blockDim.x) {
            const int d = t0 + u;
            tm[u] = make_int4(m[3 * d], m[3 * d + 1], m[3 * d + 2], 0);
            const double4 c = coef[d];
            tc[u][0] = c.x; tc[u][1] = c.y; tc[u][2] = c.z;
            tc[u][3] = rho[2 * d]; tc[u][4] = rho[2 * d + 1];
        }
        __syncthreads();
        for (int u = 0; u < nt; ++u) {
            const int mm[3] = {tm[u].x, tm[u].y, tm[u].z};
            double sn, cs;
            if (F32) {
                float s32, c32;
                phase_sincos_f(mm, v, ttab, s32, c32);
                sn = s32; cs = c32;
            } else {
                phase_sincos_d(mm, sx, sy, sz, sn, cs);
            }
            const double g = tc[u][4] * cs - tc[u][3] * sn;   // Im(e^{-i k.r} rho)
            gx += tc[u][0] * g;
            gy += tc[u][1] * g;
            gz += tc[u][2] * g;
        }
    }
    if (act) {
        F[3 * i] = q[i] * gx;
        F[3 * i + 1] = q[i] * gy;
        F[3 * i + 2] = q[i] * gz;
    }
}

size_t lrs_workspace(int nD)
{
    return (((size_t)nD * sizeof(double4) + 255) / 256) * 256 + (size_t)nD * 7 * sizeof(double) + 8 * sizeof(double);
}

cudaError_t lr_force_stateless(const double *r, const double *q, int n, const double box[3], const int *m,
                               const int *cr, const int *cnr, int nD, const double *rho, int P, double Sr,
                               double Snr, double ke, double *F, double *est, void *work, int precision,
                               cudaStream_t st)
{
    double4 *coef = static_cast<double4 *>(work);
    double *terms = reinterpret_cast<double *>(static_cast<char *>(work) + (((size_t)nD * sizeof(double4) + 255) / 256) * 256);
    double *sums = terms + (size_t)nD * 7;
    k_lrs_coef<<<(nD + 127) / 128, 128, 0, st>>>(m, cr, cnr, rho, nD, box[0], box[1], box[2], P, Sr, Snr, ke,
                                                 coef, terms);
    if (n > 0) {
        if (precision == 1)
            k_lrs_force<true><<<(n + kLrsThreads - 1) / kLrsThreads, kLrsThreads, 0, st>>>(
                r, q, n, box[0], box[1], box[2], m, rho, coef, nD, F);
        else
            k_lrs_force<false><<<(n + kLrsThreads - 1) / kLrsThreads, kLrsThreads, 0, st>>>(
                r, q, n, box[0], box[1], box[2], m, rho, coef, nD, F);
    }
    if (est) {
        k_lrs_sum<<<1, 32, 0, st>>>(terms, nD, sums);
        cudaMemcpyAsync(est, sums, 7 * sizeof(double), cudaMemcpyDeviceToHost, st);
    }
    return cudaGetLastError();
}

}  // namespace rbsog
