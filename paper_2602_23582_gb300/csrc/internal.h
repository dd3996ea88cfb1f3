// internal.h -- host-side launchers of the RBSOG kernels (one per .cu file).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace rbsog {

// Constants of the SOG split, passed by value (kernel parameter space).
struct SogConsts {
    int M, ME;                  // Gaussians of force/pressure, energy
    double rc, ke;
    double w[kMaxGauss], s[kMaxGauss], wt[kMaxGauss], st[kMaxGauss];
    // FP32 copies for the FP32 build's exclusion terms: w~_l, w_l, 1/s~_l^2, 1/s_l^2
    float wtf[kMaxGauss], wf[kMaxGauss], ist2f[kMaxGauss], is2f[kMaxGauss];
};

constexpr int kTail = 7;        // energy: degree (in u = r^2) of the Taylor tail of the wide Gaussians
constexpr int kTailF = 5;       // force: degree of its polynomial tail (Chebyshev-node interpolant)

// FP32 pair kernel constants.  The wider Gaussians vary little over r <= r_c
// and are summed as a polynomial in u = r^2: for the force, those with
// s~_l >= 1.3 r_c (u / s~^2 <= 0.6) as the degree-5 polynomial through their
// sum at the Chebyshev nodes of [0, r_c^2] (within 1e-8 of the sum at u = 0,
// 1e-7 with the FP32 rounding of its evaluation, as for the degree-8 Taylor
// polynomial it replaced; measured), for the energy those with s_l >= 2.5 r_c
// as a Taylor polynomial (remainder below 0.16^8 / 8! of w_l); the narrower
// ones are exponentials.  The energy path keeps its coefficients
// as FP32 hi + lo pairs: a rounding shared by every pair would otherwise be
// multiplied by sum q_i q_j / r, which is far larger than the short-range
// energy itself.
struct PairConstsF {
    int M, ME;
    int nff, nfe;               // exponentials for the force (l < nff) and the energy (l < nfe)
    float rc2, ke;
    float rc2_hi, rc2_lo;       // r_c^2 (1 +- 1e-5): pairs in between are decided in FP64 (with energies)
    float rl2_hi;               // (r_c + skin)^2 (1 + 1e-5): the list build's radius
    double rc2d;                // r_c^2 in FP64
    float beta[kMaxGauss];      // log2(e) / s~_l^2 (force)
    float wt[kMaxGauss];        // w~_l
    float tt[kTailF + 1];       // sum_{nff <= l < M} w~_l e^{-u / s~_l^2} ~= sum_k tt[k] u^k
    float be_hi[kMaxGauss], be_lo[kMaxGauss];   // log2(e) / s_l^2 (energy)
    float w_hi[kMaxGauss], w_lo[kMaxGauss];     // w_l
    float te[kTail + 1];        // energy tail without its constant (te[0] = 0)
    double te0;                 // sum_{nfe <= l < ME} w_l, applied in FP64 to the per-atom sum of q_i q_j
};

constexpr int kTailD = 20;      // FP64: degree (in u = r^2) of the Taylor tail of the wider Gaussians

// FP64 pair kernel constants.  Gaussians with s_l >= 0.8 r_c are summed as
// one Taylor polynomial in u = r^2 of degree kTailD (u / s_l^2 <= 1.6 for
// r <= r_c; over r <= r_c the polynomial differs from the exponentials by
// less than 2e-15 of their sum, rounding included, for Table 2 row 2 at r_c =
// 10 A: measured against direct evaluation); the nf narrower ones, of the
// force and the energy split alike (s = s~ for l < M), as exponentials.
struct PairConstsD {
    int M, ME, nf;
    double rc2, ke;
    float rc2f;                 // r_c^2 (1 + 1e-5): the FP32 candidate test
    double inv_s2[kMaxGauss];   // 1 / s_l^2
    double wt[kMaxGauss];
    double w[kMaxGauss];
    double tt[kTailD + 1];      // sum_{nf <= l < M} w~_l e^{-u/s~_l^2} = sum_k tt[k] u^k
    double te[kTailD + 1];      // sum_{nf <= l < ME} w_l e^{-u/s_l^2} = sum_k te[k] u^k
};
constexpr double kFix2Scale = 1099511627776.0;   // FP64 pair forces: two words, units 2^-40 and 2^-80

// Everything a kernel needs about the batch of systems.
struct Batch {
    int S;                      // systems
    int N;                      // atoms
    int C;                      // total cells (capacity)
    int sub;                    // cells per cutoff
    double rc;
    double rlist;               // list radius r_c + skin (cells of rlist / sub)
    int skin;                   // 1: NPT steps keep the lists while displacements allow
    DevSys *sys;                // [S]
    const int *atom_sys;        // [N]
    const int *cell_sys;        // [C]
    const int *chunk_sys, *chunk_a0, *chunk_n;   // atom chunks
    int nchunks;
    int item_cap;               // pair work items, all systems
    const int *item_sys;        // [item_cap] system of each work item index
};

// FP32 pair kernel: work items are clusters of kClus consecutive cell-sorted
// atoms of one cell; one warp per (cluster, dz plane of the half stencil),
// kCpWarps warps per block, one pair record per warp.
constexpr int kCpWarps = 4;
constexpr int kF64Split = 4;    // FP64 pair kernel: warps per (work item, dz plane), each over every 4th cell
// warps per work item of the pair kernels: FP32, one (cells of r_c: the two
// dz planes of the half stencil together, 14 cells) or sub + 1 (cells of
// r_c / sub: one dz plane each); FP64, the sub + 1 planes x kF64Split cell
// quarters
__host__ __device__ inline int pair_parts(int precision, int sub) { return precision == 1 ? (sub == 1 ? 1 : sub + 1) : (sub + 1) * kF64Split; }
// pair records per work item, as a fraction num / den (one per warp in both
// builds; the fraction leaves room for records per block)
inline int pair_rec_num(int precision, int sub) { return pair_parts(precision, sub); }
inline int pair_rec_den(int) { return 1; }

struct AtomArrays {
    double *r, *p, *F;          // [3N]
    const double *q, *mass;     // [N]
    const int *type, *mol;      // [N]
    int *cell;                  // [N]
    int *rank;                  // [N] rank in its cell after binning; cell-sorted position after sorting
    float4 *locf;               // [N] cell-local coords + mol bits (FP32)
    double4 *locd;              // [N] cell-local coords + q (FP64)
    uint4 *su;                  // [N] fixed-point fractional coords + q bits
    double *xref;               // [3N] positions at the last list build
    int *count, *start;         // [C], [C + 1]
    int *sidx;                  // [N] cell-sorted original index
    float4 *pos4;               // [kClus item_cap] FP32: cluster slots (x, y, z, molecule id), padded
    float2 *qt;                 // [kClus item_cap] FP32: cluster slots (q, type bits), padded
    double4 *posd;              // [N] sorted, FP64
    int2 *aux;                  // [N] sorted (mol, type)
    int2 *items;                // [item_cap] (cell, group) pair work items; FP32: (cell, k) = cluster k of the cell
    int2 *ccl;                  // [C] FP32: (item of the first cluster, clusters) of each cell
    float4 *cbox;               // [2 item_cap] FP32: cluster bounding box (centre | first atom, half extent | atoms)
    unsigned long long *ffix;   // pair forces, cell-sorted, fixed point: FP32 [3 N] x | y | z in units of
                                // 2^-32 (kFixScale); FP64 [6 N] x | y | z in units of 2^-40, then the
                                // remainders x | y | z in units of 2^-80 (kFix2Scale)
    float4 *posf;               // [N] FP64 build: cell-sorted cell-local coordinates in FP32 + molecule id
    // LJ table: system s owns entries [lj0, lj0 + ntypes^2) (DevSys), entry
    // ti * ntypes + tj = (4 eps sig^12, 4 eps sig^6); ljf_lo: FP32 remainders
    const float2 *ljf, *ljf_lo;
    const double2 *ljd;
    // FP64 build: (cos, sin)(2 pi k / 512), k < 512, made once by launch_turn_table_d
    // and copied into shared memory by the k-space kernels
    const double2 *turn_tab_d;
};

// ---- k_bin.cu
void launch_box_prep(const Batch &b, cudaStream_t st);
void launch_clear_flags(const Batch &b, cudaStream_t st);
// bins the atoms of the systems whose lists are rebuilt (all, outside NPT
// steps with a skin); zero_counts: clear the cell counts first
void launch_bin(const Batch &b, const AtomArrays &a, int precision, cudaStream_t st, bool zero_counts = true);
// cell-local coordinates (pos4) and fixed-point coordinates (su) of the atoms
// of systems that keep their lists, in the cells of the last build
void launch_refresh(const Batch &b, const AtomArrays &a, cudaStream_t st);
// marks every system's lists stale (positions or box set from the host)
void launch_invalidate_lists(const Batch &b, cudaStream_t st);
void launch_scan(const Batch &b, const AtomArrays &a, int precision, cudaStream_t st);
// scatter + per-cell sort (FP32: along the snake path of sub-columns, and
// the cluster bounding boxes of the rebuilt systems)
void launch_scatter_sort(const Batch &b, const AtomArrays &a, int precision, cudaStream_t st);
// FP32, lists with a skin: cluster bounding boxes of the systems that keep
// their lists (after launch_refresh)
void launch_cluster_box(const Batch &b, const AtomArrays &a, cudaStream_t st);

// ---- k_pair.cu: partial = per record (FP32: one per block of kCpWarps
// warps; FP64: one per block of kPairWarps work units = item x dz plane):
// (Ucoul, Ulj, Wc[6], Wl[6], W[6]) as kPairRec doubles; energies and the
// Coulomb/LJ split only when `energy` is set (W, the total, always).  Each
// system's item range is a multiple of kItemAlign items, so a block never
// mixes systems.  launch_reduce_pair (k_integrate.cu) sums each system's
// records into kPairRedBlocks records in a fixed order.
constexpr int kPairWarps = 1;       // FP64: one warp per block, no block-level wait on a slower warp
constexpr int kItemAlign = kCpWarps;
static_assert(kItemAlign % kPairWarps == 0, "item alignment");
constexpr int kPairRec = 20;
constexpr int kPairRedBlocks = 64;  // second-stage reduction of the unit records, per system
// records of system s: [item0 * num / den, ceil((item0 + nitems) * num / den))
void launch_reduce_pair(const Batch &b, int rec_num, int rec_den, const double *pair_part, double *pair_red,
                        cudaStream_t st);
void launch_pair(const Batch &b, const AtomArrays &a, int precision, const PairConstsF &cf,
                 const PairConstsD &cd, int energy, double *partial, cudaStream_t st);

// ---- k_sampler.cu
constexpr int kGL = 20;         // Gauss-Legendre nodes per axis of the proposal mass of a tilted cell
struct SamplerArgs {
    int P, M, kind;
    uint64_t seed;
    double wt[kMaxGauss], st[kMaxGauss];
    double cr[kMaxGauss], cn[kMaxGauss], st2q[kMaxGauss];
    double sig_u;
    double glx[kGL], glw[kGL];  // Gauss-Legendre nodes and weights on [-1, 1]
    double *tri_tab;            // lattice-sum tables of the tilted systems (SampScratch::tab0)
    int has_tri;                // 1: some system of the context has a tilted cell
};
// per-system sampler scratch: 1D lattice sums T0, T2, T4 per Gaussian and
// axis, and the chain's start state (paper MH sampler).  A tilted system
// (DevSys::tri) has instead sums over Z^3, made once for its fixed cell:
// tS[l][a] = sum_m k_a^2 e_l(m), the normalizer terms tHr, tHnr, and tables
// at tri_tab + tab0: Gy[l][a][i][j] = sum over m_2 of k_a^2 e_l (m_0 = i -
// tmm[0], m_1 = j - tmm[1]), then Gx[l][a][i] = sum over j of Gy, then
// scratch G4[l][i][j] = sum over m_2 of k^4 e_l.
struct SampScratch {
    double T[3][kMaxGauss][3];
    double start_w, start_g;
    int start_m[4];
    double tS[kMaxGauss][3], tHr[kMaxGauss], tHnr[kMaxGauss];
    long long tab0;
    int tmm[4];
};
// doubles of the tables of one tilted system (see SampScratch)
inline size_t tri_tab_size(int M, const int mm[3])
{
    const size_t nx = 2 * mm[0] + 1, ny = 2 * mm[1] + 1;
    return (size_t)M * nx * ny * 4 + (size_t)M * 3 * nx;
}
// the sums of the tilted systems (once per cell: the cell is held fixed)
void launch_tri_tables(const Batch &b, const SamplerArgs &sa, SampScratch *ss, const int *tri_sys, int ntri,
                       const int *mm_max, cudaStream_t st);
// adv = 1: the evaluation of an NPT step (counter DevSys::step + 1); 0: re-evaluate at DevSys::step
void launch_sampler(const Batch &b, const SamplerArgs &sa, int adv, int *mr, int *mnr, int *D, int *cr,
                    int *cnr, int4 *pm, double *pw, double *pg, double *pu, double *pun, SampScratch *ss,
                    int Dcap, cudaStream_t st);

// ---- k_kspace.cu
// FP64 build: the structure factor takes sub-chunks of kChunk / kSkSubD atoms
// per block (partials [chunk][sub][Dcap][2]), and the long-range force
// kLrGroupsD groups of modes per atom, each into its own partial force [3N]
// that the force assembly adds in group order.  A system of a few thousand
// atoms then spreads its FP64 k-space work over many SMs instead of one per
// chunk; the counts are fixed, so a system's sums run in the same order in
// any batch.  The FP32 build keeps one of each.
constexpr int kSkSubD = 8;
constexpr int kLrGroupsD = 8;
inline int sk_sub(int precision) { return precision == 1 ? 1 : kSkSubD; }
inline int lr_groups(int precision) { return precision == 1 ? 1 : kLrGroupsD; }
// the FP64 phase table of the k-space kernels (512 entries), filled once
void launch_turn_table_d(double2 *tab, cudaStream_t st);
constexpr int kTurnTabEntries = 512;
// part: [nchunks x sk_sub(precision) x Dcap x 2]
void launch_sk(const Batch &b, const AtomArrays &a, int precision, const int *D, int Dcap,
               double *part, cudaStream_t st);
void launch_estimate(const Batch &b, const int *first_chunk, const int *nchunk_sys, const int *D,
                     const int *cr, const int *cnr, int Dcap, int P, double ke, const double *part,
                     double *rho, ModeCoef *coef, double *est, cudaStream_t st, int precision);
// mode groups of k_estimate: est holds S x estimate_blocks(Dcap) x 7 partial sums
int estimate_blocks(int Dcap);
// V P^F,nr by the shared-proposal estimator (sec. 3.2) over the modes of the
// last evaluation: out[S x 9] (row-major 3 x 3, kcal/mol)
void launch_nr_shared(const Batch &b, const int *D, const int *cr, const double *rho, int Dcap, int P, double ke,
                      const SamplerArgs &sa, double *out, cudaStream_t st);
size_t sk_stateless_workspace(int n, int nD);
// k_sk_static.cu: a fixed scratch for the allocation-free variant
constexpr size_t kSkStaticBytes = (size_t)4 << 20;
cudaError_t sk_static_scratch(void **ptr);
cudaError_t sk_stateless(const double *r, const double *q, int n, const double box[3], const int *m,
                         int nD, double *rho, void *work, int precision, cudaStream_t st);
// long-range force on n atoms from given structure factors (eq. f_approx),
// and (est != null, host) U^F* and V P^F,nr* (xx yy zz xy xz yz)
size_t lrs_workspace(int nD);
cudaError_t lr_force_stateless(const double *r, const double *q, int n, const double box[3], const int *m,
                               const int *cr, const int *cnr, int nD, const double *rho, int P, double Sr,
                               double Snr, double ke, double *F, double *est, void *work, int precision,
                               cudaStream_t st);

// ---- k_mol.cu
struct MolArrays {
    int nmol;
    const int *mol_start, *mol_n;       // [nmol]
    const int *b_start, *a_start, *e_start;   // [nmol + 1] CSR of bonds / angles / exclusions
    const int *bonds;  const double *bk, *br0;
    const int *angles; const double *ak, *at0;
    const int *excl;
    const int *mol_sys;                 // [nmol]
    const int *mchunk_sys, *mchunk_m0, *mchunk_n;
    int nmchunks;
};
// Fmol: per-atom forces of the molecule terms, added to (zeroed by the caller)
// energy = 0: the FP32 build leaves out the exclusion energy (forces and
// virials are computed either way)
void launch_mol(const Batch &b, const AtomArrays &a, const MolArrays &m, const SogConsts &sc, double *Fmol,
                double *partial /* per mol chunk: Ue, Ub, Ua, W[6] excl, W[6] bonded */, int precision,
                int energy, cudaStream_t st);

// ---- k_integrate.cu
struct IntegArgs {
    double dt, T, Pext, gamma, gamma_box, kB, ftm2v, nktv2p;
    double c_atom, c_box;             // exp(-gamma dt), exp(-gamma_box dt)
    double ke;                        // Coulomb constant
    const double *inv_m, *sdv;        // per atom: 1 / m, sqrt((1 - c^2) m kB T ftm2v)
    int noise_f32;                    // 1: Gaussian noise drawn in FP32 (FP32 build)
    uint64_t seed;                    // a step uses the Philox counter DevSys::step + 1
};
// prep = 1: also the cell grid of the new box (k_box_prep's work)
// count (optional): zeroes the C cell counts in the same launch
void launch_box_half(const Batch &b, const IntegArgs &ia, const double *sysred, int prep, cudaStream_t st,
                     int *count = nullptr);
// bin = 1: also k_bin's work for the updated atoms (counts zeroed by the caller)
// skin (with bin = 0): flag the system for a list rebuild when an atom has
// moved beyond the step's displacement bound
void launch_atom_update(const Batch &b, const AtomArrays &a, const IntegArgs &ia, int bin, int precision,
                        cudaStream_t st, int skin = 0);
constexpr int kKinSplit = 8;   // kinetic partials per atom chunk (one per force-assembly block)
// long-range force per atom (eq. f_approx) into Flr [lr_groups(precision) x 3N]
// (FP32: beside the pair kernel)
void launch_lr_fourier(const Batch &b, const AtomArrays &a, int precision, const ModeCoef *coef, int Dcap,
                       double *Flr, cudaStream_t st);
// F = pair partials + Flr (its groups in order) + Fmol (molecule terms; null: none), then (kick != 0)
// the second half kick p += dt/2 F, and the kinetic tensor per kChunk /
// kKinSplit atoms: kin_part[chunk][kKinSplit][6] = sum p (x) p / m
void launch_force_assembly(const Batch &b, const AtomArrays &a, int precision, const double *Flr,
                           const double *Fmol, const IntegArgs &ia, int kick, double *kin_part, cudaStream_t st);
// per-system reduction of every partial into sysred[S x kRed]; advances *step
constexpr int kRed = 64;
void launch_finalize(const Batch &b, const double *pair_part, const double *est, int est_blocks, int P,
                     const double *mol_part, const int *mchunk_first, const int *mchunk_count,
                     const double *kin_part, const int *chunk_first, const int *chunk_count,
                     const double *self_energy, const IntegArgs &ia, int do_box_kick, int adv,
                     double *sysred, cudaStream_t st);
// DevSys::step = step for every system
void launch_set_step(const Batch &b, unsigned long long step, cudaStream_t st);
cudaError_t prepare_sampler(int P);
cudaError_t prepare_pair();

}  // namespace rbsog
