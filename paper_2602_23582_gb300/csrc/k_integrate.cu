// k_integrate.cu -- Langevin NPT integrator (paper eq. Langevin_NPT, Algorithm 1
// step 8) for an orthorhombic h whose coupled axes share one box momentum, and
// the per-system reductions of every partial sum.
//
// Splitting (BAOAB; the paper defers its integrator to another work, so this
// is our reading), per step n:
//   B  p^h += dt/2 G(K, W) ftm2v;   p += dt/2 F ftm2v
//   A  dt/2 exact drift: L' = L + v tau, r' = (L'/L) r + (p/m) tau, p' = (L/L') p
//   O  p <- c p + sqrt((1 - c^2) m kB T ftm2v) xi, c = exp(-gamma dt); same for p^h
//   A  dt/2 drift; wrap r into [0, L)
//   force evaluation (counter n)
//   B  p += dt/2 F ftm2v;  K = sum p (x) p / m;  p^h += dt/2 G(K, W) ftm2v
// with the generalised box force G_g = sum_{a in g} (K_aa + W_aa - P_ext V - kB T) / L_a.
#include <algorithm>

#include "internal.h"

namespace rbsog {

namespace {

__device__ __forceinline__ int axis_group(int coupling, int a)
{
    if (coupling == 0) return 0;
    if (coupling == 1) return a == 2 ? 1 : 0;
    return a;
}

__device__ void box_muller2(uint64_t a, uint64_t b, double &z0, double &z1)
{
    double u1 = u01(a), u2 = u01(b);
    double rr = sqrt(-2.0 * log(u1));
    double ang = kTwoPi * u2;
    z0 = rr * cos(ang);
    z1 = rr * sin(ang);
}

__device__ void box_force(const DevSys &d, const double *red, const IntegArgs &ia, double G[3])
{
    const double V = d.L[0] * d.L[1] * d.L[2];
    const double pext = ia.Pext / ia.nktv2p;
    G[0] = G[1] = G[2] = 0.0;
    for (int a = 0; a < 3; ++a) {
        // red: W total at [9 + a], K at [45 + a] (diagonal entries)
        double Kaa = red[45 + a], Waa = red[9 + a];
        G[axis_group(d.coupling, a)] += (Kaa + Waa - pext * V - ia.kB * ia.T) / d.L[a];
    }
}

}  // namespace

// Box part of B (first half), A, O, A.  One warp per system: lane a < 3
// works on axis a and lane g < ng on box group g, so the FP64 chains of the
// three axes (divisions, the Gaussian of each group) run side by side.  Each
// value is formed by the same operations as in a one-thread loop over axes.
constexpr int kBoxWarps = 4;

__global__ void __launch_bounds__(32 * kBoxWarps)
k_box_half(DevSys *sys, int S, const IntegArgs ia, const double *__restrict__ sysred, int prep_sub, double rc,
           double rlist, int skin, int *__restrict__ count, int C)
{
    // the cell counts of the step's binning start at zero (count: null to keep them)
    if (count)
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < C; k += gridDim.x * blockDim.x) count[k] = 0;
    const int s = blockIdx.x * kBoxWarps + (threadIdx.x >> 5), lane = lane_id();
    if (s >= S) return;
    DevSys &d = sys[s];
    if (live_n(d) == 0) {                     // empty or finished slot (warp-uniform)
        if (prep_sub > 0 && lane < 3) { d.ncell[lane] = 2 * prep_sub + 1; d.w[lane] = 1.0; }
        if (prep_sub > 0 && lane == 0) d.rebuild = 1;
        return;
    }
    const double *red = sysred + (size_t)s * kRed;
    const int ng = d.coupling == 0 ? 1 : (d.coupling == 1 ? 2 : 3);
    // O's Gaussian for group g = lane: z[g] of one Box-Muller pair per two
    // groups.  It depends on the counters only, so it is formed first, on
    // every lane without branches, and its FP64 chain (log, sqrt, sincos)
    // overlaps the box force and the first half kick below.
    uint64_t wds[4];
    draw4(ia.seed, d.rng_id, d.step + 1, PUR_BOX, 0, wds);
    double zg, sdv;
    {
        const int gz = lane < 3 ? lane : 0;
        const uint64_t wa = gz < 2 ? wds[0] : wds[2], wb = gz < 2 ? wds[1] : wds[3];
        const double rr = sqrt(-2.0 * log(u01(wa)));
        double sn, cs;
        sincos(kTwoPi * u01(wb), &sn, &cs);
        zg = rr * (gz == 1 ? sn : cs);
        const double ch = ia.c_box;
        sdv = sqrt((1.0 - ch * ch) * d.Mbox[gz] * ia.kB * ia.T * ia.ftm2v);
    }
    const int ax = lane < 3 ? lane : 0;
    const int g_of = axis_group(d.coupling, ax);            // this lane's axis -> its group
    const double La = d.L[ax];
    // generalised box force (box_force): the axis terms added per group in axis order
    double term = 0.0;
    {
        const double V = d.L[0] * d.L[1] * d.L[2];
        const double pext = ia.Pext / ia.nktv2p;
        term = (red[45 + ax] + red[9 + ax] - pext * V - ia.kB * ia.T) / La;
    }
    const double t0 = __shfl_sync(0xffffffffu, term, 0), t1 = __shfl_sync(0xffffffffu, term, 1),
                 t2 = __shfl_sync(0xffffffffu, term, 2);
    const int gg = lane < 3 ? lane : 0;                     // this lane's group
    double G = 0.0;
    if (axis_group(d.coupling, 0) == gg) G += t0;
    if (axis_group(d.coupling, 1) == gg) G += t1;
    if (axis_group(d.coupling, 2) == gg) G += t2;
    const double Mb = d.Mbox[gg];
    double ph = d.ph[gg];
    if (gg < ng && Mb > 0.0) ph += 0.5 * ia.dt * G * ia.ftm2v;
    const double tau = 0.5 * ia.dt;
    // A: the axis velocity from its group's momentum
    const double phg = __shfl_sync(0xffffffffu, ph, g_of), Mg = __shfl_sync(0xffffffffu, Mb, g_of);
    const double v1 = Mg > 0.0 ? phg / Mg : 0.0;
    const double Lp = La, Lh = La + v1 * tau;
    // O: the group's momentum with its Gaussian (formed above)
    if (gg < ng && Mb > 0.0) ph = ia.c_box * ph + sdv * zg;
    // A: second half drift with the new momentum
    const double phn = __shfl_sync(0xffffffffu, ph, g_of);
    const double v2 = Mg > 0.0 ? phn / Mg : 0.0;
    const double Ln = Lh + v2 * tau;
    if (lane < ng) d.ph[lane] = ph;
    if (lane < 3) {
        d.Lp[lane] = Lp;
        d.Lh[lane] = Lh;
        d.L[lane] = Ln;
        d.sc1[lane] = Lh / Lp;
        d.sc2[lane] = Ln / Lh;
        d.isc1[lane] = Lp / Lh;
        d.isc2[lane] = Lh / Ln;
        d.invL[lane] = 1.0 / Ln;
    }
    if (prep_sub > 0) {
        // the cell grid of the new box (as k_box_prep, cells of rlist / sub),
        // so that the atom update can bin its atoms
        bool bad = false;
        int n = 0;
        if (lane < 3) n = axis_cells(d.tri ? perp_width(d.L, d.tilt, lane) : Ln, prep_sub, rlist, d.ncap[lane], &bad);
        const bool anybad = __any_sync(0xffffffffu, bad);
        const bool regrid = __any_sync(0xffffffffu, lane < 3 && n != d.ncell[lane]);
        // lists with a skin stay valid while every displacement since the
        // build, after the affine rescaling lambda_a = L_a / Lref_a, is below
        // (min_a lambda_a rlist - r_c) / 2: a pair at least rlist apart then
        // stays at least r_c apart
        const double lam = lane < 3 ? Ln / d.Lref[lane] : 1e300;
        const double lmin = fmin(__shfl_sync(0xffffffffu, lam, 0),
                                 fmin(__shfl_sync(0xffffffffu, lam, 1), __shfl_sync(0xffffffffu, lam, 2)));
        if (lane < 3) {
            d.ncell[lane] = n;
            d.w[lane] = Ln / n;
            // tilt per cell (a tilted cell is held fixed: Ln = L)
            const int nn = __shfl_sync(0x7u, n, lane == 0 ? 1 : 2);
            d.tw[lane] = d.tri ? d.tilt[lane] / nn : 0.0;
        }
        const double L0 = __shfl_sync(0xffffffffu, Ln, 0), L1 = __shfl_sync(0xffffffffu, Ln, 1),
                     L2 = __shfl_sync(0xffffffffu, Ln, 2);
        if (lane == 0) {
            if (anybad) d.flags |= FLAG_BOX;
            d.V = L0 * L1 * L2;
            const double thr = 0.5 * (lmin * rlist - rc);
            const bool keep = skin && d.list_valid && !regrid && thr > 0.0;   // NaN lmin: rebuild
            d.thr2 = keep ? thr * thr : 0.0;
            d.rebuild = keep ? 0 : 1;
        }
    }
}

void launch_box_half(const Batch &b, const IntegArgs &ia, const double *sysred, int prep, cudaStream_t st,
                     int *count)
{
    const int g = std::max((b.S + kBoxWarps - 1) / kBoxWarps, count ? (b.C + 32 * kBoxWarps * 8 - 1) / (32 * kBoxWarps * 8) : 1);
    k_box_half<<<g, 32 * kBoxWarps, 0, st>>>(b.sys, b.S, ia, sysred, prep ? b.sub : 0, b.rc, b.rlist, b.skin, count, b.C);
}

// Atom part of B (first half), A, O, A and the wrap.  Per-system drift
// scalings come from k_box_half; 1/m and the noise amplitude are per-atom
// constants.  NF32: the Gaussian noise is drawn in FP32 (FP32 build), else in
// FP64 (Box-Muller on the same Philox words as the CPU reference).
// BIN: the updated atom is binned right away (as k_bin; the caller zeroed the
// cell counts and set the new cell grid in k_box_half).
// SKIN: the atom's displacement since the last list build, after the affine
// rescaling of the box, is checked against the step's bound (k_box_half); a
// larger one flags the system for a list rebuild.
template <bool NF32, bool BIN, bool SKIN>
__global__ void k_atom_update(DevSys *__restrict__ sys, const int *__restrict__ atom_sys, int N,
                              double *__restrict__ r, double *__restrict__ p, const double *__restrict__ F,
                              const IntegArgs ia, const AtomArrays aa, int precision)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool live = false;
    if (i < N) {
        const DevSys &ds = sys[atom_sys[i]];
        live = i - ds.atom0 < live_n(ds);     // slots hold up to their capacity
        if (BIN && !live) aa.cell[i] = -1;
    }
    const unsigned act = BIN ? __ballot_sync(0xffffffffu, live) : 0u;
    if (!live) return;
    const int s = atom_sys[i];
    const DevSys &d = sys[s];
    const double im = ia.inv_m[i], tau = 0.5 * ia.dt, kick = 0.5 * ia.dt * ia.ftm2v;
    double x[3], v[3];
    for (int a = 0; a < 3; ++a) {
        x[a] = r[3 * i + a];
        v[a] = p[3 * i + a] + kick * F[3 * i + a];
    }
    for (int a = 0; a < 3; ++a) {
        x[a] = d.sc1[a] * x[a] + v[a] * im * tau;
        v[a] = v[a] * d.isc1[a];
    }
    uint64_t wds[4];
    draw4(ia.seed, d.rng_id, d.step + 1, PUR_ATOM, (uint64_t)(i - d.atom0), wds);
    double z[4];
    if (NF32) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float u1 = ((float)(wds[2 * k] >> 40) + 0.5f) * 5.9604644775390625e-8f;   // 2^-24
            const float u2 = ((float)(wds[2 * k + 1] >> 40) + 0.5f) * 5.9604644775390625e-8f;
            const float rr = sqrtf(-2.f * logf(u1));
            float sn, cs;
            sincospif(2.f * u2, &sn, &cs);
            z[2 * k] = (double)(rr * cs);
            z[2 * k + 1] = (double)(rr * sn);
        }
    } else {
        box_muller2(wds[0], wds[1], z[0], z[1]);
        box_muller2(wds[2], wds[3], z[2], z[3]);
    }
    const double c = ia.c_atom, sdv = ia.sdv[i];
    for (int a = 0; a < 3; ++a) v[a] = c * v[a] + sdv * z[a];
    for (int a = 0; a < 3; ++a) {
        x[a] = d.sc2[a] * x[a] + v[a] * im * tau;
        v[a] = v[a] * d.isc2[a];
        if (!d.tri) {
            const double L = d.L[a];
            x[a] -= L * floor(x[a] * d.invL[a]);
            if (x[a] >= L) x[a] -= L;
            if (x[a] < 0.0) x[a] += L;
        }
        p[3 * i + a] = v[a];
    }
    if (d.tri) {
        // into the tilted cell by whole cell vectors: x - h floor(h^{-1} x)
        double sf[3], n[3];
        frac_of(d, x, sf);
        for (int a = 0; a < 3; ++a) n[a] = floor(sf[a]);
        sub_lattice(d, n, x);
    }
    for (int a = 0; a < 3; ++a) r[3 * i + a] = x[a];
    if (SKIN && !d.rebuild) {
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double u = x[a] - aa.xref[3 * i + a] * (d.L[a] / d.Lref[a]);
            u -= d.L[a] * rint(u * d.invL[a]);
            d2 += u * u;
        }
        if (!(d2 <= d.thr2)) sys[s].rebuild = 1;   // every far atom writes the same value
    }
    if (BIN) bin_atom(d, i, x, aa.q[i], aa.mol[i], act, aa.cell, aa.rank, aa.count, aa.locf, aa.locd, aa.su, precision, true);
}

void launch_atom_update(const Batch &b, const AtomArrays &a, const IntegArgs &ia, int bin, int precision,
                        cudaStream_t st, int skin)
{
    // blocks of 256: with blocks of 128 (every SM busy) the water step measured
    // 5.6 us faster with the L2 warm but 37 us slower with it flushed between
    // steps (the atom update then overlaps the sampler's FP64 kernels longer)
    const int g = (b.N + 255) / 256;
#define RBSOG_ATOM_UPDATE(NF, BN, SK) \
    k_atom_update<NF, BN, SK><<<g, 256, 0, st>>>(b.sys, b.atom_sys, b.N, a.r, a.p, a.F, ia, a, precision)
    if (ia.noise_f32) {
        if (bin) RBSOG_ATOM_UPDATE(true, true, false);
        else if (skin) RBSOG_ATOM_UPDATE(true, false, true);
        else RBSOG_ATOM_UPDATE(true, false, false);
    } else {
        if (bin) RBSOG_ATOM_UPDATE(false, true, false);
        else if (skin) RBSOG_ATOM_UPDATE(false, false, true);
        else RBSOG_ATOM_UPDATE(false, false, false);
    }
#undef RBSOG_ATOM_UPDATE
}

// Per-system reduction of all partials (fixed order) into sysred[s][kRed]:
//  [0..8] energies (RBSOG_E_*), [9..14] W total (xx yy zz xy xz yz),
//  [15..20] W short Coulomb, [21..26] W^F,r*, [27..32] W^F,nr*, [33..38] W LJ,
//  [39..44] W bonded + exclusions, [45..50] K, [51] V, [52..54] L,
//  [55] nD, [56] acc r, [57] acc nr, [58] flags, [59..61] box momenta.
// Second stage of the pair records: system s's records (rec_num / rec_den per
// active item: FP32, one per block of kCpWarps (item, plane) warps; FP64, one
// per (dz plane, cell quarter)) in kPairRedBlocks contiguous ranges, each
// summed in a fixed order.
// grid (S, kPairRedBlocks).
constexpr int kRedThreads = 128;

__global__ void __launch_bounds__(kRedThreads)
k_reduce_pair(const DevSys *__restrict__ sys, int rec_num, int rec_den, const double *__restrict__ part,
              double *__restrict__ red)
{
    __shared__ double buf[kPairRec * (kRedThreads + 1) + 4 * kPairRec];
    const int s = blockIdx.x;
    const DevSys &d = sys[s];
    const long long u0 = (long long)d.item0 * rec_num / rec_den;   // item0 is a multiple of rec_den
    const int nu = (int)(((long long)d.nitems * rec_num + rec_den - 1) / rec_den);
    const int per = (nu + kPairRedBlocks - 1) / kPairRedBlocks;
    const int a = min(nu, (int)blockIdx.y * per), e = min(nu, a + per);
    double v[kPairRec];
#pragma unroll
    for (int k = 0; k < kPairRec; ++k) v[k] = 0.0;
    for (int r = a + threadIdx.x; r < e; r += kRedThreads) {
        const double *pp = part + (size_t)(u0 + r) * kPairRec;
#pragma unroll
        for (int k = 0; k < kPairRec; ++k) v[k] += pp[k];
    }
    block_reduce_lanes<kPairRec, kRedThreads>(v, buf, red + ((size_t)s * kPairRedBlocks + blockIdx.y) * kPairRec);
}

void launch_reduce_pair(const Batch &b, int rec_num, int rec_den, const double *pair_part, double *pair_red,
                        cudaStream_t st)
{
    k_reduce_pair<<<dim3(b.S, kPairRedBlocks), kRedThreads, 0, st>>>(b.sys, rec_num, rec_den, pair_part, pair_red);
}

constexpr int kFinThreads = 128;

__global__ void __launch_bounds__(kFinThreads)
k_finalize(DevSys *sys, const double *__restrict__ pair_part, const double *__restrict__ est, int est_blocks,
           int P, const double *__restrict__ mol_part, const int *__restrict__ mchunk_first,
           const int *__restrict__ mchunk_count, const double *__restrict__ kin_part,
           const int *__restrict__ chunk_first, const int *__restrict__ chunk_count,
           const double *__restrict__ self_energy, const IntegArgs ia, int do_box_kick, int adv,
           double *__restrict__ sysred, int span)
{
    constexpr int NV = kPairRec + 21;   // pair records + 15 molecule + 6 kinetic partial sums
    __shared__ double buf[NV * (kFinThreads + 1) + 4 * NV];
    __shared__ double acc[NV];
    const int s = blockIdx.x, tid = threadIdx.x;
    DevSys &d = sys[s];
    if (!d.act) return;                       // empty or finished: keep the last results
    double *o = sysred + (size_t)s * kRed;
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    // pair records, already reduced to kPairRedBlocks per system
    for (int c = tid; c < kPairRedBlocks; c += blockDim.x) {
        const double *pp = pair_part + ((size_t)s * kPairRedBlocks + c) * kPairRec;
#pragma unroll
        for (int k = 0; k < kPairRec; ++k) v[k] += pp[k];
    }
    constexpr int M0 = kPairRec, K0 = kPairRec + 15;
    for (int c = tid; c < mchunk_count[s]; c += blockDim.x) {
        const double *pp = mol_part + (size_t)(mchunk_first[s] + c) * 15;
#pragma unroll
        for (int k = 0; k < 15; ++k) v[M0 + k] += pp[k];
    }
    for (int c = tid; c < chunk_count[s] * kKinSplit; c += blockDim.x) {
        const double *pp = kin_part + ((size_t)chunk_first[s] * kKinSplit + c) * 6;
#pragma unroll
        for (int k = 0; k < 6; ++k) v[K0 + k] += pp[k];
    }
    block_reduce_lanes<NV, kFinThreads>(v, buf, acc);
    __syncthreads();
    if (tid >= 32) return;
    // the outputs on the lanes of warp 0 (short FP64 chains side by side);
    // every value is formed by the same operations as in a one-thread loop
    const int lane = tid;
    // long range (eqs. U_F*, P_F,r*, P_F,nr*): mode-group sums in group order
    // (lane t < 7), then the prefactors k_e S^r / (4 V P) and -k_e S^nr / (8 V P)
    double es = 0.0;
    if (lane < 7)
        for (int g = 0; g < est_blocks; ++g) es += est[((size_t)s * est_blocks + g) * 7 + lane];
    const double Vb = d.L[0] * d.L[1] * d.L[2];
    const double lrl = lane == 0 ? ia.ke * d.Sr / (4.0 * Vb * P) * es : -ia.ke * d.Snr / (8.0 * Vb * P) * es;
    const double lr0 = __shfl_sync(0xffffffffu, lrl, 0);
    const int a = lane < 6 ? lane : 0;
    const double Wnr = __shfl_sync(0xffffffffu, lrl, 1 + a);
    const double us = self_energy[2 * s];        // U_self (App. A)
    const double uxc = self_energy[2 * s + 1];   // FP32 build: sum over exclusions of ke q_i q_j F_E(0)
    // energies and the Coulomb/LJ virial split come from the pair kernel only
    // on energy steps (zero otherwise); the total short-range virial always
    double e[9];
    e[0] = acc[0];                 // U^N Coulomb
    e[1] = lr0;                    // U^F*
    e[2] = us;
    e[3] = acc[M0] - uxc;          // exclusions
    e[4] = acc[1];                 // LJ
    e[5] = acc[M0 + 1];            // bonds
    e[6] = acc[M0 + 2];            // angles
    e[7] = e[0] + e[1] - e[2] + e[3];
    e[8] = 0.5 * (acc[K0] + acc[K0 + 1] + acc[K0 + 2]);
    // tensor component a on lane a < 6
    const double K = acc[K0 + a];
    const double Wc = acc[2 + a], Wl = acc[8 + a];
    const double Wr = a < 3 ? lr0 : 0.0;
    const double Wb = acc[M0 + 3 + a] + acc[M0 + 9 + a];
    const double W = acc[14 + a] + Wr + Wnr + Wb;
    bool finite = true;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        if (lane == k) o[k] = e[k];
        finite = finite && isfinite(e[k]);
    }
    if (lane < 6) {
        o[9 + a] = W; o[15 + a] = Wc; o[21 + a] = Wr; o[27 + a] = Wnr;
        o[33 + a] = Wl; o[39 + a] = Wb; o[45 + a] = K;
    }
    finite = __all_sync(0xffffffffu, finite && (lane >= 6 || isfinite(W)));
    // second half of the box kick: generalised box force (box_force) on lanes
    // a < 3, added per group in axis order
    const int ng = d.coupling == 0 ? 1 : (d.coupling == 1 ? 2 : 3);
    const double pext = ia.Pext / ia.nktv2p;
    const double term = (K + W - pext * Vb - ia.kB * ia.T) / d.L[a];
    const double t0 = __shfl_sync(0xffffffffu, term, 0), t1 = __shfl_sync(0xffffffffu, term, 1),
                 t2 = __shfl_sync(0xffffffffu, term, 2);
    const int gg = lane < 3 ? lane : 0;
    double ph = d.ph[gg];
    if (do_box_kick && d.n > 0 && lane < ng && d.Mbox[gg] > 0.0) {
        double G = 0.0;
        if (axis_group(d.coupling, 0) == gg) G += t0;
        if (axis_group(d.coupling, 1) == gg) G += t1;
        if (axis_group(d.coupling, 2) == gg) G += t2;
        ph += 0.5 * ia.dt * G * ia.ftm2v;
        d.ph[gg] = ph;
    }
    const double ph0 = __shfl_sync(0xffffffffu, ph, 0), ph1 = __shfl_sync(0xffffffffu, ph, 1),
                 ph2 = __shfl_sync(0xffffffffu, ph, 2);
    if (lane != 0) return;
    if (!finite) d.flags |= FLAG_NONFINITE;
    o[51] = Vb;
    o[52] = d.L[0]; o[53] = d.L[1]; o[54] = d.L[2];
    o[55] = d.nD; o[56] = d.nacc_r; o[57] = d.nacc_nr; o[58] = d.flags;
    o[59] = ph0; o[60] = ph1; o[61] = ph2;
    if (adv) {
        d.step += 1ull;
        if (d.steps_left > 0 && --d.steps_left == 0) d.act = 0;   // the last requested step
    }
    o[62] = (double)d.step;
    o[63] = (double)d.list_builds;
}

__global__ void k_set_step(DevSys *sys, int S, unsigned long long step)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) sys[s].step = step;
}

void launch_set_step(const Batch &b, unsigned long long step, cudaStream_t st)
{
    k_set_step<<<(b.S + 127) / 128, 128, 0, st>>>(b.sys, b.S, step);
}

void launch_finalize(const Batch &b, const double *pair_part, const double *est, int est_blocks, int P,
                     const double *mol_part,
                     const int *mchunk_first, const int *mchunk_count, const double *kin_part,
                     const int *chunk_first, const int *chunk_count, const double *self_energy,
                     const IntegArgs &ia, int do_box_kick, int adv, double *sysred, cudaStream_t st)
{
    k_finalize<<<b.S, kFinThreads, 0, st>>>(b.sys, pair_part, est, est_blocks, P, mol_part, mchunk_first, mchunk_count,
                                            kin_part, chunk_first, chunk_count, self_energy, ia, do_box_kick,
                                            adv, sysred, 2 * b.sub + 1);
}

}  // namespace rbsog
