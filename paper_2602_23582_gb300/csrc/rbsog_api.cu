// rbsog_api.cu -- the C ABI (include/rbsog.h): context set-up, one force
// evaluation (Algorithm 1 steps 2-7), Langevin NPT steps as a replayed CUDA
// graph (step 8), checkpoints and introspection.
//
// Launch sequence of one evaluation on the context stream, with the mode
// sampler forked onto a second stream (it needs only the box):
//   box_prep -> [fork: sampler] -> bin -> scan -> scatter+sort -> pair ->
//   [join] -> S(k) -> estimate -> long-range force -> molecules ->
//   kick/kinetic -> finalize (+ step counter advance)
// An NPT step prepends box_half and atom_update.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rbsog.h"
#include "internal.h"

using namespace rbsog;

namespace {

constexpr double kKB = 0.0019872067;                         // kcal/(mol K)
constexpr double kFtm2v = 1.0 / 48.88821291 / 48.88821291;   // (kcal/mol/A)/(g/mol) -> A/fs^2
constexpr double kNktv2p = 68568.415;                        // atm per kcal/(mol A^3)

// Capacities of one slot of a context: a fixed batch sizes them by its
// systems, a pool by the caller's slot classes.
struct SlotCaps {
    int atoms = 0, mols = 0, bonds = 0, angles = 0, excl = 0, types = 1;
    double rho = 0.0;                  // atoms per A^3 the slot's FP32 pair lists are sized for
    double box[3] = {0.0, 0.0, 0.0};   // largest box the slot's cell grid is sized for
};

// Where a slot's data lives in the context's arrays.
struct SlotLayout {
    SlotCaps caps;
    int atom0 = 0, mol0 = 0, bond0 = 0, angle0 = 0, excl0 = 0, lj0 = 0;
};

// Host image of one system in its slot (global indices already applied).
struct SlotImage {
    std::vector<double> r, p, q, mass, inv_m, sdv;
    std::vector<int> type, mol;
    std::vector<int> b_start, a_start, e_start;   // nmol + 1
    std::vector<int> bonds, angles, excl;
    std::vector<double> bk, br0, ak, at0;
    std::vector<double2> ljd;
    std::vector<float2> ljf, ljf_lo;
    double self_e[2] = {0.0, 0.0};
};

}  // namespace

struct rbsog_ctx {
    rbsog_params prm{};
    std::vector<SlotLayout> lay;        // per slot
    std::vector<double> sog_w;          // w_l (energy split), for per-system constants
    bool pool = false;                  // slots are loaded and emptied at run time
    std::vector<rbsog_status> slot_err; // pool: why a slot's system was stopped (RBSOG_OK: it was not)
    int S = 0, N = 0, C = 0, Dcap = 0, nchunks = 0, nmol = 0, nmchunks = 0, item_cap = 0;
    cudaStream_t st = nullptr, st2 = nullptr, st3 = nullptr;   // st2: mode sampling, st3: molecule terms
    cudaStream_t st4 = nullptr;         // records the pair-kernel trace events beside the main stream
    bool own_st = false, own_st2 = false;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fork3 = nullptr, ev_join3 = nullptr;
    cudaEvent_t ev_fork4 = nullptr, ev_join4 = nullptr, ev_bin = nullptr;
    cudaEvent_t ev_tr[3] = {nullptr, nullptr, nullptr};   // forks to / join from st4
    std::string err;
    std::vector<int> h_atom0, h_n, h_cell0, h_ncap_total, h_coupling;
    std::vector<double> h_tilt;         // per system (xy, xz, yz): tilted cells are held fixed
    double *tri_tab = nullptr;          // lattice-sum tables of the tilted systems
    std::vector<void *> allocs;
    // device
    DevSys *sys = nullptr;
    double *r = nullptr, *p = nullptr, *F = nullptr, *q = nullptr, *mass = nullptr;
    double *Fmol = nullptr;     // molecule-term forces, added by the force assembly
    double *Flr = nullptr;      // long-range forces [lr_groups x 3N] (FP32: beside the pair kernel), added by the force assembly
    int *type = nullptr, *mol = nullptr, *atom_sys = nullptr, *cell = nullptr, *rank = nullptr;
    float4 *locf = nullptr, *pos4 = nullptr;
    double4 *locd = nullptr, *posd = nullptr;
    uint4 *su = nullptr;
    double *xref = nullptr;   // positions at the last list build
    int *count = nullptr, *start = nullptr, *sidx = nullptr, *cell_sys = nullptr;
    int *item_sys = nullptr;
    float2 *qt = nullptr;
    int2 *aux = nullptr, *items = nullptr;
    int *chunk_sys = nullptr, *chunk_a0 = nullptr, *chunk_n = nullptr, *first_chunk = nullptr, *nchunk_sys = nullptr;
    int *mchunk_sys = nullptr, *mchunk_m0 = nullptr, *mchunk_n = nullptr, *mchunk_first = nullptr, *mchunk_count = nullptr;
    int *b_start = nullptr, *a_start = nullptr, *e_start = nullptr, *bonds = nullptr, *angles = nullptr, *excl = nullptr;
    double *bk = nullptr, *br0 = nullptr, *ak = nullptr, *at0 = nullptr;
    double *pair_part = nullptr, *est = nullptr, *mol_part = nullptr, *kin_part = nullptr, *sysred = nullptr;
    double *self_e = nullptr;
    float4 *posf = nullptr;     // FP64 build: cell-sorted coordinates in FP32 (candidate tests)
    unsigned long long *ffix = nullptr;   // pair forces in fixed point (FP32: 3 N words, FP64: 6 N)
    int2 *ccl = nullptr;        // FP32 build: per cell (first cluster item, clusters)
    float4 *cbox = nullptr;     // FP32 build: cluster bounding boxes
    double *pair_red = nullptr; // pair records reduced to kPairRedBlocks per system
    double *inv_m = nullptr, *sdv = nullptr;   // per-atom integrator constants
    double2 *ljd = nullptr;     // LJ blocks per system
    double2 *turn_tab_d = nullptr;   // FP64 build: the k-space kernels' phase table
    float2 *ljf = nullptr, *ljf_lo = nullptr;
    int *mr = nullptr, *mnr = nullptr, *D = nullptr, *cr = nullptr, *cnr = nullptr;
    int4 *pm = nullptr;
    SampScratch *samp = nullptr;
    double *nrsh = nullptr;     // [S x 9] shared-proposal estimator output
    double *pw = nullptr, *pg = nullptr, *pu = nullptr, *pun = nullptr;
    double *sk_part = nullptr, *rho = nullptr;
    ModeCoef *coef = nullptr;
    // launch descriptions
    Batch b{};
    AtomArrays a{};
    MolArrays m{};
    PairConstsF pcf{};
    PairConstsD pcd{};
    SogConsts sc{};
    SamplerArgs sa{};
    IntegArgs ia{};
    // graphs of one NPT step: [0] forces and virial, [1] also energies
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    cudaGraph_t graph_src[2] = {nullptr, nullptr};
    cudaGraphExec_t eval_graph[2] = {nullptr, nullptr};   // one evaluation: [0] force only, [1] with energies
    cudaGraph_t eval_graph_src[2] = {nullptr, nullptr};
    // pair-kernel trace: event-record nodes around the pair kernel in each
    // graph; their events are swapped per launch to a ring of caller-visible
    // timings (placeholders when no trace is armed)
    cudaEvent_t ev_pair_ph[2] = {nullptr, nullptr};
    cudaGraphNode_t pair_node[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    bool pair_node_live[2] = {false, false};
    std::vector<cudaEvent_t> ring_s, ring_e;
    int ring_pos = 0;
    unsigned long long h_step = 0;   // host copy of the device step counter
    // timing
    bool timing = false;
    bool mol_late = false;    // molecule terms joined before the force assembly (FP32 build, large molecules)
    std::vector<std::string> t_names;
    std::vector<cudaEvent_t> t_events;
    std::vector<double> t_ms;
};

namespace {

thread_local std::string g_create_err;   // error text of a failed rbsog_create

// Radius of the pair lists and of the cells (r_c + skin; the skin applies to
// the FP32 build only).
double list_radius(const rbsog_params &P)
{
    return P.rc + (P.precision == RBSOG_FP32 ? P.skin : 0.0);
}

rbsog_status fail(rbsog_ctx *c, rbsog_status s, const std::string &msg)
{
    if (c) c->err = msg;
    g_create_err = msg;
    return s;
}

rbsog_status cuda_fail(rbsog_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, RBSOG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// every cudaMalloc and cudaFree the library makes (rbsog_debug_device_alloc_calls)
std::atomic<unsigned long long> g_dev_alloc_calls{0};

template <typename T>
bool dalloc(rbsog_ctx *c, T *&ptr, size_t n)
{
    if (n == 0) n = 1;
    void *v = nullptr;
    ++g_dev_alloc_calls;
    if (cudaMalloc(&v, n * sizeof(T)) != cudaSuccess) return false;
    cudaMemset(v, 0, n * sizeof(T));
    c->allocs.push_back(v);
    ptr = static_cast<T *>(v);
    return true;
}

template <typename T>
bool upload(rbsog_ctx *c, T *&ptr, const std::vector<T> &h)
{
    if (!dalloc(c, ptr, h.size())) return false;
    if (!h.empty() && cudaMemcpy(ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return false;
    return true;
}

// SOG terms of sec. 2.2 / 3.1 (omega rescales l = 0 in both splits)
void sog_terms(const rbsog_params &p, int M, std::vector<double> &w, std::vector<double> &s,
               std::vector<double> &wt, std::vector<double> &st)
{
    w.resize(M); s.resize(M); wt.resize(M); st.resize(M);
    const double c = std::sqrt(2.0 / kPi), lb = std::log(p.b);
    for (int l = 0; l < M; ++l) {
        double bl = std::pow(p.b, (double)l);
        s[l] = std::sqrt(2.0) * bl * p.sigma;
        st[l] = s[l];
        w[l] = c * lb / (p.sigma * bl);
        wt[l] = c * lb / (bl * bl * bl * p.sigma * p.sigma * p.sigma);
    }
    w[0] *= p.omega;
    wt[0] *= p.omega;
}

// Sampler constants (the same expressions as the paper's formulas, FP64 on
// the host): pi^1.5 w~ s~^5 and pi^1.5 w~ s~^7 (eqs. samplingP,
// samplingPnr), s~^2 / 4, and the proposal's standard deviation (App. D).
void fill_sampler_args(const rbsog_params &P, const std::vector<double> &wt, const std::vector<double> &st,
                       SamplerArgs &sa)
{
    sa.P = P.P; sa.M = P.M; sa.kind = P.sampler; sa.seed = P.seed;
    const double pi15 = std::pow(kPi, 1.5);
    for (int l = 0; l < P.M; ++l) {
        double s5 = st[l] * st[l] * st[l] * st[l] * st[l];
        sa.wt[l] = wt[l]; sa.st[l] = st[l];
        sa.cr[l] = pi15 * wt[l] * s5;
        sa.cn[l] = pi15 * wt[l] * s5 * st[l] * st[l];
        sa.st2q[l] = st[l] * st[l] * 0.25;
    }
    sa.sig_u = 1.0 / (std::sqrt(2.0) * kPi * st[0]);
    // Gauss-Legendre rule of kGL nodes on [-1, 1]: the roots of P_n by Newton
    // iteration from cos(pi (i + 3/4) / (n + 1/2)), weights 2 / ((1 - x^2) P_n'(x)^2)
    const int n = kGL;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double x = std::cos(kPi * (i + 0.75) / (n + 0.5)), dpn = 1.0;
        for (int it = 0; it < 100; ++it) {
            double pm1 = 1.0, pn = x;                 // P_0, P_1
            for (int k = 2; k <= n; ++k) {
                const double pk = ((2 * k - 1) * x * pn - (k - 1) * pm1) / k;
                pm1 = pn;
                pn = pk;
            }
            dpn = n * (x * pn - pm1) / (x * x - 1.0);
            const double step = pn / dpn;
            x -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        double pm1 = 1.0, pn = x;
        for (int k = 2; k <= n; ++k) {
            const double pk = ((2 * k - 1) * x * pn - (k - 1) * pm1) / k;
            pm1 = pn;
            pn = pk;
        }
        dpn = n * (x * pn - pm1) / (x * x - 1.0);
        sa.glx[i] = -x;
        sa.glx[n - 1 - i] = x;
        sa.glw[i] = sa.glw[n - 1 - i] = 2.0 / ((1.0 - x * x) * dpn * dpn);
    }
    sa.tri_tab = nullptr;
    sa.has_tri = 0;
}

// Range |m_a| <= mm[a] of the lattice sums of a tilted cell: the box around
// the ellipsoid |k| <= 2 sqrt(46) / s~_0 (beyond it every term is below
// e^-46 of the largest), |m_a| <= (2 sqrt(46) / (2 pi s~_0)) |a-th cell vector|.
void tri_range(const double L[3], const double t[3], double st0, int mm[3])
{
    const double R = 2.0 * std::sqrt(46.0) / st0 / (2.0 * kPi);
    const double len[3] = {L[0], std::sqrt(t[0] * t[0] + L[1] * L[1]), std::sqrt(t[1] * t[1] + t[2] * t[2] + L[2] * L[2])};
    for (int a = 0; a < 3; ++a) mm[a] = (int)std::ceil(R * len[a]) + 2;
}

bool tilted(const rbsog_system_desc &d) { return d.tilt[0] != 0.0 || d.tilt[1] != 0.0 || d.tilt[2] != 0.0; }

// the extent that sets the cell grid along axis a: the edge, or for a tilted
// cell its perpendicular width
double grid_span(const rbsog_system_desc &d, int a) { return perp_width(d.box, d.tilt, a); }

void record(rbsog_ctx *c, const char *name)
{
    if (!c->timing) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, c->st);
    c->t_events.push_back(e);
    c->t_names.push_back(name);
}

// One force evaluation of every system (Algorithm 1 steps 2-7).
// adv = 1: the evaluation of an NPT step (Philox counter DevSys::step + 1,
// advanced at the end); 0: evaluate at DevSys::step.
// Mode sampling on the second stream: needs the box and its cell grid only.
// Unless kernels are timed one by one, the structure factor and the estimator
// follow on the same stream (fork_kspace) and the join comes after them.
void fork_sampler(rbsog_ctx *c, int adv)
{
    cudaEventRecord(c->ev_fork, c->st);
    cudaStreamWaitEvent(c->st2, c->ev_fork, 0);
    launch_sampler(c->b, c->sa, adv, c->mr, c->mnr, c->D, c->cr, c->cnr, c->pm, c->pw, c->pg, c->pu, c->pun,
                   c->samp, c->Dcap, c->st2);
    if (c->timing) cudaEventRecord(c->ev_join, c->st2);
}

// Structure factor, estimator and long-range force on the second stream,
// after the sampler and the binning (which writes the fixed-point coordinates
// they read): they need neither the cell lists nor the pair forces, so they
// run beside the list build and the pair evaluation.
void enqueue_kspace(rbsog_ctx *c, cudaStream_t st)
{
    launch_sk(c->b, c->a, c->prm.precision, c->D, c->Dcap, c->sk_part, st);
    record(c, "structure_factor");
    launch_estimate(c->b, c->first_chunk, c->nchunk_sys, c->D, c->cr, c->cnr, c->Dcap, c->prm.P, c->prm.ke,
                    c->sk_part, c->rho, c->coef, c->est, st, c->prm.precision);
    record(c, "estimate");
    // FP32 build: the long-range force too.  In the FP64 build it is FP64 work
    // like the pair kernel's, and beside it measured slower than after it
    // (water: pair 1.42 -> 1.81 ms, step 1.87 -> 2.29 ms): it follows the join.
    if (c->prm.precision == RBSOG_FP32 || c->timing) {
        launch_lr_fourier(c->b, c->a, c->prm.precision, c->coef, c->Dcap, c->Flr, st);
        record(c, "lr_force");
    }
}

void fork_kspace(rbsog_ctx *c)
{
    if (c->timing) return;
    cudaEventRecord(c->ev_bin, c->st);
    cudaStreamWaitEvent(c->st2, c->ev_bin, 0);
    enqueue_kspace(c, c->st2);
    cudaEventRecord(c->ev_join, c->st2);
}

// Molecule terms on the third stream: they need only the positions and the
// box and run beside the binning into their own force buffer.  In the FP32
// build, and for large molecules (a warp each, e.g. 15-site ions with 137
// terms) in both builds, they join before the force assembly and overlap the
// pair kernel (water, FP32: the step 0.203 -> 0.198 ms, the pair launch
// unchanged; joined before the pair kernel they held it back).  Small
// molecules in the FP64 build join before the pair kernel: their FP64 bonded
// terms would share the FP64 pipe with it.
void fork_mol(rbsog_ctx *c, int energy)
{
    if (c->m.nmchunks == 0) return;
    cudaEventRecord(c->ev_fork3, c->st);
    cudaStreamWaitEvent(c->st3, c->ev_fork3, 0);
    cudaMemsetAsync(c->Fmol, 0, 3 * sizeof(double) * (size_t)c->N, c->st3);
    launch_mol(c->b, c->a, c->m, c->sc, c->Fmol, c->mol_part, c->prm.precision, energy, c->st3);
    cudaEventRecord(c->ev_join3, c->st3);
}

// prepared = 1: the caller has set the cell grid, binned the atoms and
// forked the sampler and the molecule terms (the NPT step does this in its
// box and atom updates).
void enqueue_eval(rbsog_ctx *c, int kick, int box_kick, int energy, int adv, int prepared = 0)
{
    const int prec = c->prm.precision;
    const bool mol = c->m.nmchunks > 0;
    if (!prepared) {
        record(c, "start");
        fork_mol(c, energy);
        launch_box_prep(c->b, c->st);
        record(c, "box_prep");
        fork_sampler(c, adv);
        launch_bin(c->b, c->a, prec, c->st);
        record(c, "bin");
    }
    fork_kspace(c);
    launch_scan(c->b, c->a, prec, c->st);
    record(c, "scan");
    launch_scatter_sort(c->b, c->a, prec, c->st);
    record(c, "scatter_sort");
    if (mol && !c->mol_late) cudaStreamWaitEvent(c->st, c->ev_join3, 0);
    // in a graph capture: event-record nodes at the pair kernel's start and end
    // (external records, retargeted per launch by arm_pair_trace), on st4: an
    // event node between two kernels of the main stream would stand between
    // them and their programmatic (early-launch) edge
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->st, &cap);
    const bool trace = cap == cudaStreamCaptureStatusActive && c->ev_pair_ph[0] && c->ev_pair_ph[1];
    if (trace) {
        cudaEventRecord(c->ev_tr[0], c->st);
        cudaStreamWaitEvent(c->st4, c->ev_tr[0], 0);
        cudaEventRecordWithFlags(c->ev_pair_ph[0], c->st4, cudaEventRecordExternal);
    }
    launch_pair(c->b, c->a, prec, c->pcf, c->pcd, energy, c->pair_part, c->st);
    if (trace) {
        cudaEventRecord(c->ev_tr[1], c->st);
        cudaStreamWaitEvent(c->st4, c->ev_tr[1], 0);
        cudaEventRecordWithFlags(c->ev_pair_ph[1], c->st4, cudaEventRecordExternal);
        cudaEventRecord(c->ev_tr[2], c->st4);
    }
    record(c, "pair");
    // the pair records are reduced beside the long-range part
    cudaEventRecord(c->ev_fork4, c->st);
    cudaStreamWaitEvent(c->st3, c->ev_fork4, 0);
    launch_reduce_pair(c->b, pair_rec_num(prec, c->prm.cell_sub), pair_rec_den(prec), c->pair_part, c->pair_red,
                       c->st3);
    cudaEventRecord(c->ev_join4, c->st3);
    cudaStreamWaitEvent(c->st, c->ev_join, 0);
    record(c, "sampler_join");
    if (c->timing) enqueue_kspace(c, c->st);
    if (mol && c->mol_late) cudaStreamWaitEvent(c->st, c->ev_join3, 0);
    if (prec != RBSOG_FP32 && !c->timing) launch_lr_fourier(c->b, c->a, prec, c->coef, c->Dcap, c->Flr, c->st);
    launch_force_assembly(c->b, c->a, prec, c->Flr, mol ? c->Fmol : nullptr, c->ia, kick, c->kin_part, c->st);
    record(c, "assembly_kick");
    cudaStreamWaitEvent(c->st, c->ev_join4, 0);
    if (trace) cudaStreamWaitEvent(c->st, c->ev_tr[2], 0);   // st4 joins (long done by now)
    launch_finalize(c->b, c->pair_red, c->est, estimate_blocks(c->Dcap), c->prm.P, c->mol_part, c->mchunk_first, c->mchunk_count, c->kin_part,
                    c->first_chunk, c->nchunk_sys, c->self_e, c->ia, box_kick, adv, c->sysred, c->st);
    record(c, "finalize");
}

void enqueue_npt_step(rbsog_ctx *c, int energy)
{
    // box half-step with the new cell grid, the sampler forked right after
    // it, then the atom update with the binning of the moved atoms
    launch_box_half(c->b, c->ia, c->sysred, 1, c->st, c->count);
    fork_sampler(c, 1);
    if (c->b.skin) {
        // lists with a skin: the atom update flags the systems that rebuild,
        // which are then binned; the others get their coordinates in the
        // cells of their last build
        launch_atom_update(c->b, c->a, c->ia, 0, c->prm.precision, c->st, 1);
        launch_bin(c->b, c->a, c->prm.precision, c->st, false);
        launch_refresh(c->b, c->a, c->st);
        launch_cluster_box(c->b, c->a, c->st);
    } else {
        launch_atom_update(c->b, c->a, c->ia, 1, c->prm.precision, c->st);
    }
    fork_mol(c, energy);
    enqueue_eval(c, 1, 1, energy, 1, 1);
}

// The status flags of a host copy h of the systems' records: the first
// failing system's error (a pool stops that system only and goes on).
rbsog_status process_flags(rbsog_ctx *c, std::vector<DevSys> &h)
{
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < c->S; ++s) {
        if (!h[s].flags) continue;
        rbsog_status st = RBSOG_OK;
        std::string why;
        if (h[s].flags & FLAG_BOX) {
            st = RBSOG_EBOX;
            why = "box edge below " + std::to_string(2 * c->prm.cell_sub + 1) + " cells of r_c/sub";
        } else if (h[s].flags & FLAG_OVERFLOW) {
            st = RBSOG_EOVERFLOW;
            why = "a cell holds more than " + std::to_string(kCellCap) + " atoms";
        } else {
            st = RBSOG_ENONFINITE;
            why = "non-finite energy or virial";
        }
        if (!c->pool) return fail(c, st, "system " + std::to_string(s) + ": " + why);
        // a pool stops the failing system only; the others go on
        if (c->slot_err[s] == RBSOG_OK) c->slot_err[s] = st;
        h[s].act = 0;
        h[s].flags = 0;
        e = cudaMemcpy(c->sys + s, &h[s], sizeof(DevSys), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(c, e, "device");
    }
    return RBSOG_OK;
}

rbsog_status check_flags(rbsog_ctx *c)
{
    std::vector<DevSys> h(c->S);
    cudaError_t e = cudaMemcpyAsync(h.data(), c->sys, sizeof(DevSys) * c->S, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "device");
    return process_flags(c, h);
}

// 3x3 row-major from the six components xx yy zz xy xz yz
static const int kSym[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};

void results_from(rbsog_ctx *c, const std::vector<double> &h, rbsog_result *res);

rbsog_status fill_results(rbsog_ctx *c, rbsog_result *res)
{
    std::vector<double> h((size_t)c->S * kRed);
    cudaError_t e = cudaMemcpyAsync(h.data(), c->sysred, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "results");
    results_from(c, h, res);
    return RBSOG_OK;
}

// The result records from a host copy h of the per-system reductions.
void results_from(rbsog_ctx *c, const std::vector<double> &h, rbsog_result *res)
{
    const int *sym = kSym;
    for (int s = 0; s < c->S; ++s) {
        const double *o = &h[(size_t)s * kRed];
        rbsog_result &r = res[s];
        std::memset(&r, 0, sizeof(r));
        for (int k = 0; k < 9; ++k) r.energy[k] = o[k];
        for (int k = 0; k < 9; ++k) {
            r.virial[k] = o[9 + sym[k]];
            r.virial_coul_short[k] = o[15 + sym[k]];
            r.virial_long_r[k] = o[21 + sym[k]];
            r.virial_long_nr[k] = o[27 + sym[k]];
            r.virial_lj[k] = o[33 + sym[k]];
            r.virial_bonded[k] = o[39 + sym[k]];
            r.pressure[k] = (o[9 + sym[k]] + o[45 + sym[k]]) / o[51] * kNktv2p;
        }
        r.volume = o[51];
        r.box[0] = o[52]; r.box[1] = o[53]; r.box[2] = o[54];
        for (int a = 0; a < 3; ++a) r.tilt[a] = c->h_tilt.empty() ? 0.0 : c->h_tilt[3 * s + a];
        r.n_distinct_modes = (int)o[55];
        r.n_accept_r = (int)o[56];
        r.n_accept_nr = (int)o[57];
        r.step = (uint64_t)o[62];
        r.list_builds = (int)o[63];
    }
}

void free_ctx(rbsog_ctx *c)
{
    if (!c) return;
    for (auto g : c->graph)
        if (g) cudaGraphExecDestroy(g);
    for (auto g : c->graph_src)
        if (g) cudaGraphDestroy(g);
    for (int k = 0; k < 2; ++k) {
        if (c->eval_graph[k]) cudaGraphExecDestroy(c->eval_graph[k]);
        if (c->eval_graph_src[k]) cudaGraphDestroy(c->eval_graph_src[k]);
    }
    for (auto e : c->ring_s) cudaEventDestroy(e);
    for (auto e : c->ring_e) cudaEventDestroy(e);
    for (auto e : c->ev_pair_ph)
        if (e) cudaEventDestroy(e);
    for (auto e : c->t_events) cudaEventDestroy(e);
    for (void *v : c->allocs) {
        ++g_dev_alloc_calls;
        cudaFree(v);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_bin) cudaEventDestroy(c->ev_bin);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_fork3) cudaEventDestroy(c->ev_fork3);
    if (c->ev_join3) cudaEventDestroy(c->ev_join3);
    if (c->ev_fork4) cudaEventDestroy(c->ev_fork4);
    if (c->ev_join4) cudaEventDestroy(c->ev_join4);
    if (c->own_st2 && c->st2) cudaStreamDestroy(c->st2);
    for (auto ev : c->ev_tr)
        if (ev) cudaEventDestroy(ev);
    if (c->st3) cudaStreamDestroy(c->st3);
    if (c->st4) cudaStreamDestroy(c->st4);
    if (c->own_st && c->st) cudaStreamDestroy(c->st);
    delete c;
}

SlotCaps caps_of(const rbsog_system_desc &d)
{
    SlotCaps cp;
    cp.atoms = d.n_atoms;
    int nm = 0;
    for (int i = 0; i < d.n_atoms; ++i)
        if (i == 0 || d.mol[i] != d.mol[i - 1]) ++nm;
    cp.mols = nm;
    cp.bonds = d.n_bonds;
    cp.angles = d.n_angles;
    cp.excl = d.n_excl;
    cp.types = d.ntypes;
    for (int a = 0; a < 3; ++a) cp.box[a] = d.box[a];
    cp.rho = d.n_atoms / (d.box[0] * d.box[1] * d.box[2]);
    return cp;
}

// Image of system d for the slot `ly`; fills the per-system fields of ds
// (box, box masses, counts, Philox key word, step 0).  false + why on a
// system that does not fit the slot or is inconsistent.
bool build_image(const rbsog_params &P, const SlotLayout &ly, DevSys &ds, const rbsog_system_desc &d,
                 const std::vector<double> &w, SlotImage &im, std::string &why)
{
    const SlotCaps &cp = ly.caps;
    const int n = d.n_atoms;
    if (n > cp.atoms || d.ntypes > cp.types || d.n_bonds > cp.bonds || d.n_angles > cp.angles ||
        d.n_excl > cp.excl) {
        why = "system larger than its slot";
        return false;
    }
    for (int a = 0; a < 3; ++a) {
        const double x = std::floor(grid_span(d, a) * P.cell_sub / list_radius(P));
        if (!(x >= 2 * P.cell_sub + 1)) { why = "box edge too small for the cell stencil"; return false; }
        if (!(x <= ds.ncap[a])) { why = "box larger than its slot's cell grid"; return false; }
    }
    const double c_atom = std::exp(-P.gamma * P.dt);
    im.r.assign(d.r0, d.r0 + 3 * (size_t)n);
    im.p.resize(3 * (size_t)n);
    im.q.assign(d.q, d.q + n);
    im.mass.assign(d.mass, d.mass + n);
    im.inv_m.resize(n);
    im.sdv.resize(n);
    im.type.assign(d.type, d.type + n);
    im.mol.assign(d.mol, d.mol + n);
    double sq = 0.0;
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) im.p[3 * i + a] = d.v0 ? d.v0[3 * i + a] * d.mass[i] : 0.0;
        im.inv_m[i] = 1.0 / d.mass[i];
        im.sdv[i] = std::sqrt((1.0 - c_atom * c_atom) * d.mass[i] * kKB * P.T * kFtm2v);
        if (d.type[i] < 0 || d.type[i] >= d.ntypes) { why = "atom type out of range"; return false; }
        sq += d.q[i] * d.q[i];
    }
    // App. A: U_self = ln b / (sqrt(2 pi) sigma) (omega + (1 - b^{-(M-1)})/(b - 1)) sum q^2
    im.self_e[0] = P.ke * std::log(P.b) / (std::sqrt(2.0 * kPi) * P.sigma) *
                   (P.omega + (1.0 - std::pow(P.b, -(P.M_energy - 1.0))) / (P.b - 1.0)) * sq;
    // FP32 build: the constant part sum_excl ke q_i q_j F_E(0) of the exclusion energy
    if (P.precision == RBSOG_FP32) {
        double fe0 = 0.0, sx = 0.0;
        for (int l = 0; l < P.M_energy; ++l) fe0 += w[l];
        for (int e2 = 0; e2 < d.n_excl; ++e2) sx += d.q[d.excl[2 * e2]] * d.q[d.excl[2 * e2 + 1]];
        im.self_e[1] = P.ke * fe0 * sx;
    }
    // molecules: maximal runs of equal mol id; their term lists in molecule order
    std::vector<int> mol_of(n);
    int nm = 0;
    for (int i = 0; i < n; ++i) {
        if (i == 0 || d.mol[i] != d.mol[i - 1]) ++nm;
        mol_of[i] = nm - 1;
    }
    if (nm > cp.mols) { why = "more molecules than the slot holds"; return false; }
    std::vector<std::vector<int>> mb(nm), ma(nm), me(nm);
    auto same = [&](int i, int j) { return i >= 0 && j >= 0 && i < n && j < n && mol_of[i] == mol_of[j]; };
    for (int e2 = 0; e2 < d.n_bonds; ++e2) {
        const int i = d.bonds[2 * e2], j = d.bonds[2 * e2 + 1];
        if (!same(i, j)) { why = "a bond spans two molecules"; return false; }
        mb[mol_of[i]].push_back(e2);
    }
    for (int e2 = 0; e2 < d.n_angles; ++e2) {
        const int i = d.angles[3 * e2], j = d.angles[3 * e2 + 1], kk = d.angles[3 * e2 + 2];
        if (!same(i, j) || !same(j, kk)) { why = "an angle spans two molecules"; return false; }
        ma[mol_of[i]].push_back(e2);
    }
    for (int e2 = 0; e2 < d.n_excl; ++e2) {
        const int i = d.excl[2 * e2], j = d.excl[2 * e2 + 1];
        if (!same(i, j)) { why = "an exclusion spans two molecules"; return false; }
        me[mol_of[i]].push_back(e2);
    }
    const int A0 = ly.atom0;
    im.b_start.assign(1, ly.bond0);
    im.a_start.assign(1, ly.angle0);
    im.e_start.assign(1, ly.excl0);
    for (int mm = 0; mm < nm; ++mm) {
        for (int e2 : mb[mm]) {
            im.bonds.push_back(A0 + d.bonds[2 * e2]); im.bonds.push_back(A0 + d.bonds[2 * e2 + 1]);
            im.bk.push_back(d.bond_k[e2]); im.br0.push_back(d.bond_r0[e2]);
        }
        for (int e2 : ma[mm]) {
            for (int t = 0; t < 3; ++t) im.angles.push_back(A0 + d.angles[3 * e2 + t]);
            im.ak.push_back(d.angle_k[e2]); im.at0.push_back(d.angle_t0[e2]);
        }
        for (int e2 : me[mm]) { im.excl.push_back(A0 + d.excl[2 * e2]); im.excl.push_back(A0 + d.excl[2 * e2 + 1]); }
        im.b_start.push_back(ly.bond0 + (int)im.bk.size());
        im.a_start.push_back(ly.angle0 + (int)im.ak.size());
        im.e_start.push_back(ly.excl0 + (int)im.excl.size() / 2);
    }
    // LJ block: (4 eps sig^12, 4 eps sig^6) per type pair, FP32 hi + lo copies
    for (int t = 0; t < d.ntypes * d.ntypes; ++t) {
        const double eps = d.lj_eps[t], sg = d.lj_sig[t];
        const double s6 = sg * sg * sg * sg * sg * sg;
        im.ljd.push_back(make_double2(4.0 * eps * s6 * s6, 4.0 * eps * s6));
        im.ljf.push_back(make_float2((float)im.ljd.back().x, (float)im.ljd.back().y));
        im.ljf_lo.push_back(make_float2((float)(im.ljd.back().x - (double)im.ljf.back().x),
                                        (float)(im.ljd.back().y - (double)im.ljf.back().y)));
    }
    // per-system fields
    for (int a = 0; a < 3; ++a) { ds.L[a] = d.box[a]; ds.ph[a] = 0.0; ds.Mbox[a] = 0.0; ds.tilt[a] = d.tilt[a]; }
    ds.tri = tilted(d) ? 1 : 0;
    ds.V = d.box[0] * d.box[1] * d.box[2];
    ds.n = n;
    ds.nmol = nm;
    ds.ntypes = d.ntypes;
    ds.rng_id = d.rng_id;
    // FP32 in-cell order: sub-columns about one cluster (kClus atoms at the
    // system's density) wide
    {
        const double rho = n / (d.box[0] * d.box[1] * d.box[2]);
        const double a = std::cbrt(kClus / std::max(rho, 1e-12));
        const double wcell = list_radius(P) / P.cell_sub;
        ds.kc = std::min(4, std::max(1, (int)std::lround(wcell / a)));
        if (P.cluster_cols > 0) ds.kc = P.cluster_cols;
    }
    ds.step = 0;                      // the system's first evaluation uses counter 0
    ds.flags = 0;
    ds.steps_left = -1;
    // box masses: M_g = n_g^2 V ftm2v / (kappa L_g^2 omega^2), kappa in (kcal/mol/A^3)^-1
    if (P.coupling != RBSOG_COUPLE_FIXED && P.tau_box > 0 && P.compressibility > 0) {
        const double kap = P.compressibility * kNktv2p, om = 2.0 * kPi / P.tau_box;
        if (ds.coupling == 0) {
            ds.Mbox[0] = 9.0 * ds.V * kFtm2v / (kap * d.box[0] * d.box[0] * om * om);
        } else {
            ds.Mbox[0] = 4.0 * ds.V * kFtm2v / (kap * d.box[0] * d.box[0] * om * om);
            ds.Mbox[1] = 1.0 * ds.V * kFtm2v / (kap * d.box[2] * d.box[2] * om * om);
        }
    }
    return true;
}

rbsog_status validate_params(const rbsog_params *p)
{
    if (!p) return RBSOG_EINVAL;
    if (!(p->rc > 0) || !(p->b > 1) || !(p->sigma > 0) || p->M < 1 || p->M > kMaxGauss ||
        p->M_energy < p->M || p->M_energy > kMaxGauss || p->P < 1 || p->P > kMaxP ||
        p->sampler < 0 || p->sampler > 2 || (p->precision != 0 && p->precision != 1) ||
        (p->cell_sub < 0 || p->cell_sub > 2) || p->coupling < 0 || p->coupling > 2 || p->thermo_every < 0 ||
        !(p->skin >= 0.0 && p->skin <= p->rc) || p->cluster_cols < 0 || p->cluster_cols > 4)
        return RBSOG_EINVAL;
    return RBSOG_OK;
}

rbsog_status validate_system(const rbsog_system_desc &d)
{
    if (d.n_atoms < 1 || !d.q || !d.mass || !d.type || !d.mol || !d.r0 || d.ntypes < 1 ||
        d.ntypes > kMaxTypes || !d.lj_eps || !d.lj_sig)
        return RBSOG_EINVAL;
    if ((d.n_bonds > 0 && (!d.bonds || !d.bond_k || !d.bond_r0)) ||
        (d.n_angles > 0 && (!d.angles || !d.angle_k || !d.angle_t0)) || (d.n_excl > 0 && !d.excl) ||
        d.n_bonds < 0 || d.n_angles < 0 || d.n_excl < 0)
        return RBSOG_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(d.box[a] > 0) || !std::isfinite(d.tilt[a])) return RBSOG_EBOX;
    for (int i = 0; i < d.n_atoms; ++i)
        if (!(d.mass[i] > 0) || !std::isfinite(d.mass[i])) return RBSOG_EINVAL;
    return RBSOG_OK;
}

}  // namespace

extern "C" {

void rbsog_default_params(rbsog_params *p, double rc)
{
    std::memset(p, 0, sizeof(*p));
    p->rc = rc;
    p->b = 1.62976708826776469;          // Table 2, row 2
    p->sigma = 3.270345668108471 * rc / 9.0;
    p->omega = 1.007806979343806;
    p->M = 10;
    p->M_energy = 10;
    p->P = 100;
    p->sampler = RBSOG_SAMPLER_PAPER;
    p->seed = 1;
    p->precision = RBSOG_FP32;
    p->thermo_every = 1;
    p->ke = 332.06371;
    p->dt = 0.5;
    p->T = 300.0;
    p->P_ext = 1.0;
    p->gamma = 1.0 / 100.0;              // 0.1 ps thermostat (sec. 4.3)
    p->gamma_box = 1.0 / 500.0;          // 0.5 ps barostat
    p->tau_box = 500.0;
    p->compressibility = 4.5e-5 * 1.01325;   // 4.5e-5 bar^-1 in atm^-1
    p->coupling = RBSOG_COUPLE_ISO;
    p->cell_sub = 0;
}

const char *rbsog_last_error(const rbsog_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

unsigned long long rbsog_debug_device_alloc_calls(void) { return g_dev_alloc_calls.load(); }

int rbsog_n_atoms(const rbsog_ctx *ctx) { return ctx ? ctx->N : 0; }

rbsog_status rbsog_system_range(const rbsog_ctx *ctx, int s, int *atom0, int *n)
{
    if (!ctx || s < 0 || s >= ctx->S) return RBSOG_EINVAL;
    if (atom0) *atom0 = ctx->h_atom0[s];
    if (n) *n = ctx->h_n[s];
    return RBSOG_OK;
}

void rbsog_destroy(rbsog_ctx *ctx) { free_ctx(ctx); }

}  // extern "C"

namespace {

// A context of n slots: `systems` (one per slot, sizes exact) or, for a pool,
// `pool_caps` (empty slots of the given capacities).
rbsog_status create_impl(const rbsog_params *params, int n_systems, const rbsog_system_desc *systems,
                         const SlotCaps *pool_caps, void *stream, rbsog_ctx **out)
{
    if (!out) return RBSOG_EINVAL;
    *out = nullptr;
    rbsog_status vs = validate_params(params);
    if (vs != RBSOG_OK) return vs;
    if (n_systems <= 0 || (!systems && !pool_caps)) return RBSOG_EINVAL;
    for (int k = 0; systems && k < n_systems; ++k) {
        vs = validate_system(systems[k]);
        if (vs != RBSOG_OK) return vs;
    }
    rbsog_ctx *c = new (std::nothrow) rbsog_ctx();
    if (!c) return RBSOG_ENOMEM;
    try {
        c->prm = *params;
        c->pool = systems == nullptr;
        c->slot_err.assign(n_systems, RBSOG_OK);
        bool any_tri = false;
        for (int k = 0; systems && k < n_systems; ++k) any_tri = any_tri || tilted(systems[k]);
        if (any_tri && (c->prm.coupling != RBSOG_COUPLE_FIXED || c->prm.skin > 0.0 ||
                        c->prm.sampler != RBSOG_SAMPLER_PAPER)) {
            rbsog_status rr = fail(c, RBSOG_EUNSUPPORTED,
                                   "a tilted cell needs coupling RBSOG_COUPLE_FIXED, skin 0 and the paper sampler");
            free_ctx(c);
            return rr;
        }
        if (c->prm.cell_sub == 0) {
            // cells of r_c/2 when a box edge leaves little room above 3 r_c (the
            // box fluctuates in NPT), else cells of r_c; pools take r_c/2
            c->prm.cell_sub = c->pool ? 2 : 1;
            for (int k = 0; systems && k < n_systems; ++k)
                for (int a2 = 0; a2 < 3; ++a2)
                    if (grid_span(systems[k], a2) < 3.3 * list_radius(c->prm)) c->prm.cell_sub = 2;
        }
        const rbsog_params &P = c->prm;
        c->S = n_systems;
        c->st = static_cast<cudaStream_t>(stream);
        cudaError_t e = cudaSuccess;
        if (!c->st) {
            // the legacy default stream cannot be captured into a graph: use a
            // blocking stream of our own (it orders with the legacy stream)
            e = cudaStreamCreate(&c->st);
            if (e != cudaSuccess) { rbsog_status r = cuda_fail(c, e, "stream"); free_ctx(c); return r; }
            c->own_st = true;
        }
        e = cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking);
        if (e != cudaSuccess) { rbsog_status r = cuda_fail(c, e, "stream"); free_ctx(c); return r; }
        c->own_st2 = true;
        e = cudaStreamCreateWithFlags(&c->st3, cudaStreamNonBlocking);
        if (e != cudaSuccess) { rbsog_status r = cuda_fail(c, e, "stream"); free_ctx(c); return r; }
        e = cudaStreamCreateWithFlags(&c->st4, cudaStreamNonBlocking);
        if (e != cudaSuccess) { rbsog_status r = cuda_fail(c, e, "stream"); free_ctx(c); return r; }
        for (auto &ev : c->ev_tr) cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_bin, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_fork3, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_join3, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_fork4, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_join4, cudaEventDisableTiming);
        cudaEventCreate(&c->ev_pair_ph[0]);
        cudaEventCreate(&c->ev_pair_ph[1]);
        c->Dcap = (P.sampler == RBSOG_SAMPLER_IID) ? 2 * P.P : P.P + 1;

        // ---- host layout: one slot per system, sized by its capacities
        const int S = c->S;
        std::vector<SlotCaps> caps(S);
        for (int k = 0; k < S; ++k) {
            if (systems) caps[k] = caps_of(systems[k]);
            else caps[k] = pool_caps[k];
        }
        std::vector<double> w, s, wt, st;
        const int MM = std::max(P.M, P.M_energy);
        sog_terms(P, MM, w, s, wt, st);
        c->sog_w = w;
        std::vector<DevSys> hsys(S);
        c->lay.resize(S);
        int N = 0, C = 0, nmolx = 0, item_cap = 0, nbond = 0, nang = 0, nexc = 0, nlj = 0;
        std::vector<int> atom_sys, cell_sys, item_sys, chunk_sys, chunk_a0, chunk_n, first_chunk(S), nchunk(S);
        std::vector<int> mchunk_sys, mchunk_m0, mchunk_n, mchunk_first(S), mchunk_count(S);
        c->h_atom0.resize(S); c->h_n.resize(S); c->h_cell0.resize(S); c->h_ncap_total.resize(S);
        for (int k = 0; k < S; ++k) {
            const SlotCaps &cp = caps[k];
            DevSys &ds = hsys[k];
            std::memset(&ds, 0, sizeof(ds));
            int ncap_t = 1;
            for (int a = 0; a < 3; ++a) {
                const double span = systems ? grid_span(systems[k], a) : cp.box[a];
                const int n = (int)std::floor(span * P.cell_sub / list_radius(P));
                if (n < 2 * P.cell_sub + 1) {
                    rbsog_status rr = fail(c, RBSOG_EBOX, "system " + std::to_string(k) + ": box edge " +
                                                              std::to_string(cp.box[a]) + " too small for the cell stencil");
                    free_ctx(c);
                    return rr;
                }
                // room for the box to grow by 15% under pressure
                const int cap = (int)std::floor(cp.box[a] * 1.15 * P.cell_sub / list_radius(P));
                ds.ncap[a] = std::max(cap, n);
                ncap_t *= ds.ncap[a];
                ds.L[a] = cp.box[a];
            }
            SlotLayout &ly = c->lay[k];
            ly.caps = cp;
            ly.atom0 = N; ly.mol0 = nmolx; ly.bond0 = nbond; ly.angle0 = nang; ly.excl0 = nexc; ly.lj0 = nlj;
            ds.cell0 = C;
            ds.ncell_cap_total = ncap_t;
            // pair work items (FP32: clusters of kClus atoms; FP64: groups of
            // 32): at most one partial group per cell; a multiple of
            // kItemAlign so that no pair-kernel block spans two systems
            const int gsize = P.precision == RBSOG_FP32 ? kClus : 32;
            ds.item0 = item_cap;
            ds.item_cap = ((cp.atoms + gsize - 1) / gsize + ncap_t + kItemAlign - 1) / kItemAlign * kItemAlign;
            item_cap += ds.item_cap;
            item_sys.insert(item_sys.end(), (size_t)ds.item_cap, k);
            ds.atom0 = N;
            ds.lj0 = nlj;
            ds.mol0 = nmolx;
            ds.coupling = P.coupling == RBSOG_COUPLE_SEMI_ISO ? 1 : 0;
            ds.steps_left = -1;
            c->h_atom0[k] = N; c->h_n[k] = 0; c->h_cell0[k] = C; c->h_ncap_total[k] = ncap_t;
            for (int i = 0; i < ncap_t; ++i) cell_sys.push_back(k);
            C += ncap_t;
            for (int i = 0; i < cp.atoms; ++i) atom_sys.push_back(k);
            first_chunk[k] = (int)chunk_sys.size();
            for (int a0 = 0; a0 < cp.atoms; a0 += kChunk) {
                chunk_sys.push_back(k);
                chunk_a0.push_back(N + a0);
                chunk_n.push_back(std::min(kChunk, cp.atoms - a0));
            }
            nchunk[k] = (int)chunk_sys.size() - first_chunk[k];
            mchunk_first[k] = (int)mchunk_sys.size();
            // one thread per molecule when the slot's molecules are small on
            // average, else chunks of a few large molecules (one warp each)
            const int mch = (double)cp.bonds + cp.angles + cp.excl <= (double)kSmallTerms * cp.mols
                                ? kMolChunk : kMolChunkLarge;
            if (cp.mols > 0 && (mch == kMolChunkLarge || P.precision == RBSOG_FP32)) c->mol_late = true;
            for (int m0 = 0; m0 < cp.mols; m0 += mch) {
                mchunk_sys.push_back(k);
                mchunk_m0.push_back(nmolx + m0);
                mchunk_n.push_back(std::min(mch, cp.mols - m0));
            }
            mchunk_count[k] = (int)mchunk_sys.size() - mchunk_first[k];
            N += cp.atoms;
            nmolx += cp.mols + 1;             // + the end of the last molecule's term lists
            nbond += cp.bonds; nang += cp.angles; nexc += cp.excl; nlj += cp.types * cp.types;
        }
        if (N >= (1 << 25)) {
            // the pair kernel's queue packs a neighbour index into 25 bits
            rbsog_status rr = fail(c, RBSOG_EUNSUPPORTED, "more than 2^25 - 1 atoms in one context");
            free_ctx(c);
            return rr;
        }
        // global host arrays; empty slots keep harmless defaults
        std::vector<double> r(3 * (size_t)N, 0.0), p(3 * (size_t)N, 0.0), q(N, 0.0), mass(N, 1.0);
        std::vector<double> inv_m(N, 1.0), sdv(N, 0.0), self_e(2 * S, 0.0);
        std::vector<int> type(N, 0), mol(N, 0);
        std::vector<int> b_start(nmolx, 0), a_start(nmolx, 0), e_start(nmolx, 0);
        std::vector<int> bonds(2 * (size_t)nbond, 0), angles(3 * (size_t)nang, 0), excl(2 * (size_t)nexc, 0);
        std::vector<double> bk(nbond, 0.0), br0(nbond, 0.0), ak(nang, 0.0), at0(nang, 0.0);
        std::vector<double2> ljd(nlj, make_double2(0.0, 0.0));
        std::vector<float2> ljf(nlj, make_float2(0.f, 0.f)), ljf_lo(nlj, make_float2(0.f, 0.f));
        for (int k = 0; k < S; ++k) {
            const SlotLayout &ly = c->lay[k];
            for (int m = 0; m <= ly.caps.mols; ++m) {   // empty term lists
                b_start[ly.mol0 + m] = ly.bond0;
                a_start[ly.mol0 + m] = ly.angle0;
                e_start[ly.mol0 + m] = ly.excl0;
            }
        }
        if (systems) {
            for (int k = 0; k < S; ++k) {
                SlotImage im;
                std::string why;
                if (!build_image(P, c->lay[k], hsys[k], systems[k], w, im, why)) {
                    rbsog_status rr = fail(c, RBSOG_EINVAL, "system " + std::to_string(k) + ": " + why);
                    free_ctx(c);
                    return rr;
                }
                const SlotLayout &ly = c->lay[k];
                std::copy(im.r.begin(), im.r.end(), r.begin() + 3 * (size_t)ly.atom0);
                std::copy(im.p.begin(), im.p.end(), p.begin() + 3 * (size_t)ly.atom0);
                std::copy(im.q.begin(), im.q.end(), q.begin() + ly.atom0);
                std::copy(im.mass.begin(), im.mass.end(), mass.begin() + ly.atom0);
                std::copy(im.inv_m.begin(), im.inv_m.end(), inv_m.begin() + ly.atom0);
                std::copy(im.sdv.begin(), im.sdv.end(), sdv.begin() + ly.atom0);
                std::copy(im.type.begin(), im.type.end(), type.begin() + ly.atom0);
                std::copy(im.mol.begin(), im.mol.end(), mol.begin() + ly.atom0);
                std::copy(im.b_start.begin(), im.b_start.end(), b_start.begin() + ly.mol0);
                std::copy(im.a_start.begin(), im.a_start.end(), a_start.begin() + ly.mol0);
                std::copy(im.e_start.begin(), im.e_start.end(), e_start.begin() + ly.mol0);
                std::copy(im.bonds.begin(), im.bonds.end(), bonds.begin() + 2 * (size_t)ly.bond0);
                std::copy(im.bk.begin(), im.bk.end(), bk.begin() + ly.bond0);
                std::copy(im.br0.begin(), im.br0.end(), br0.begin() + ly.bond0);
                std::copy(im.angles.begin(), im.angles.end(), angles.begin() + 3 * (size_t)ly.angle0);
                std::copy(im.ak.begin(), im.ak.end(), ak.begin() + ly.angle0);
                std::copy(im.at0.begin(), im.at0.end(), at0.begin() + ly.angle0);
                std::copy(im.excl.begin(), im.excl.end(), excl.begin() + 2 * (size_t)ly.excl0);
                std::copy(im.ljd.begin(), im.ljd.end(), ljd.begin() + ly.lj0);
                std::copy(im.ljf.begin(), im.ljf.end(), ljf.begin() + ly.lj0);
                std::copy(im.ljf_lo.begin(), im.ljf_lo.end(), ljf_lo.begin() + ly.lj0);
                self_e[2 * k] = im.self_e[0];
                self_e[2 * k + 1] = im.self_e[1];
                hsys[k].act = 1;
                c->h_n[k] = systems[k].n_atoms;
            }
        }
        c->N = N; c->C = C; c->nmol = nmolx; c->item_cap = item_cap;
        c->nchunks = (int)chunk_sys.size();
        c->nmchunks = (int)mchunk_sys.size();

        // ---- device buffers
        bool ok = upload(c, c->sys, hsys) && upload(c, c->r, r) && upload(c, c->p, p) && upload(c, c->q, q) &&
                  upload(c, c->mass, mass) && upload(c, c->type, type) && upload(c, c->mol, mol) &&
                  upload(c, c->atom_sys, atom_sys) && upload(c, c->cell_sys, cell_sys) &&
                  upload(c, c->item_sys, item_sys) &&
                  upload(c, c->chunk_sys, chunk_sys) && upload(c, c->chunk_a0, chunk_a0) &&
                  upload(c, c->chunk_n, chunk_n) && upload(c, c->first_chunk, first_chunk) &&
                  upload(c, c->nchunk_sys, nchunk) && upload(c, c->mchunk_sys, mchunk_sys) &&
                  upload(c, c->mchunk_m0, mchunk_m0) && upload(c, c->mchunk_n, mchunk_n) &&
                  upload(c, c->mchunk_first, mchunk_first) && upload(c, c->mchunk_count, mchunk_count) &&
                  upload(c, c->b_start, b_start) && upload(c, c->a_start, a_start) && upload(c, c->e_start, e_start) &&
                  upload(c, c->bonds, bonds) && upload(c, c->angles, angles) && upload(c, c->excl, excl) &&
                  upload(c, c->bk, bk) && upload(c, c->br0, br0) && upload(c, c->ak, ak) && upload(c, c->at0, at0) &&
                  upload(c, c->self_e, self_e) && dalloc(c, c->F, 3 * (size_t)N) && dalloc(c, c->Fmol, 3 * (size_t)N) && dalloc(c, c->Flr, 3 * (size_t)N * lr_groups(P.precision)) && dalloc(c, c->cell, N) &&
                  dalloc(c, c->rank, N) && dalloc(c, c->sidx, N) && dalloc(c, c->count, C) &&
                  dalloc(c, c->start, C + 1) && dalloc(c, c->items, item_cap) &&
                  dalloc(c, c->pair_part, (size_t)item_cap * pair_rec_num(P.precision, P.cell_sub) /
                                              pair_rec_den(P.precision) * kPairRec) &&
                  dalloc(c, c->pair_red, (size_t)S * kPairRedBlocks * kPairRec) &&
                  dalloc(c, c->est, (size_t)S * estimate_blocks(c->Dcap) * 7) && dalloc(c, c->mol_part, (size_t)c->nmchunks * 15) &&
                  dalloc(c, c->kin_part, (size_t)c->nchunks * kKinSplit * 6) && dalloc(c, c->sysred, (size_t)S * kRed) &&
                  dalloc(c, c->mr, (size_t)S * P.P * 3) && dalloc(c, c->mnr, (size_t)S * P.P * 3) &&
                  dalloc(c, c->D, (size_t)S * c->Dcap * 3) && dalloc(c, c->cr, (size_t)S * c->Dcap) &&
                  dalloc(c, c->cnr, (size_t)S * c->Dcap) && dalloc(c, c->pm, (size_t)S * P.P) && dalloc(c, c->samp, (size_t)S) && dalloc(c, c->nrsh, (size_t)S * 9) &&
                  dalloc(c, c->pw, (size_t)S * P.P) && dalloc(c, c->pg, (size_t)S * P.P) &&
                  dalloc(c, c->pu, (size_t)S * P.P) && dalloc(c, c->pun, (size_t)S * P.P) &&
                  dalloc(c, c->sk_part, (size_t)c->nchunks * sk_sub(P.precision) * c->Dcap * 2) &&
                  dalloc(c, c->rho, (size_t)S * c->Dcap * 2) && dalloc(c, c->coef, (size_t)S * c->Dcap) &&
                  upload(c, c->ljd, ljd) && upload(c, c->ljf, ljf) && upload(c, c->ljf_lo, ljf_lo) &&
                  upload(c, c->inv_m, inv_m) && upload(c, c->sdv, sdv);
        if (ok) {
            if (P.precision == 1)
                ok = dalloc(c, c->locf, N) && dalloc(c, c->pos4, (size_t)kClus * (item_cap + 1)) &&
                     dalloc(c, c->qt, (size_t)kClus * (item_cap + 1)) && dalloc(c, c->su, N) &&
                     dalloc(c, c->ffix, 3 * (size_t)N) && dalloc(c, c->ccl, C) && dalloc(c, c->cbox, 2 * (size_t)item_cap);
            else
                ok = dalloc(c, c->locd, N) && dalloc(c, c->posd, N) && dalloc(c, c->aux, N) &&
                     dalloc(c, c->posf, N) && dalloc(c, c->ffix, 6 * (size_t)N) &&
                     dalloc(c, c->turn_tab_d, (size_t)kTurnTabEntries);
            if (ok && c->turn_tab_d) {
                // on the stream of dalloc's memset (the legacy default stream), after it, and
                // finished before any kernel of the context's streams reads the table
                launch_turn_table_d(c->turn_tab_d, 0);
                ok = cudaStreamSynchronize(0) == cudaSuccess && cudaGetLastError() == cudaSuccess;
            }
            ok = ok && dalloc(c, c->xref, 3 * (size_t)N);
        }
        if (ok && P.precision == 1) {
            // the dummy cluster past the last item (the FP32 pair kernel's
            // empty tiles): far-away atoms of no molecule
            std::vector<float4> far(kClus, make_float4(1e15f, 1e15f, 1e15f, 0.f));
            int m2 = -2;
            for (auto &f : far) std::memcpy(&f.w, &m2, sizeof(int));
            ok = cudaMemcpy(c->pos4 + (size_t)kClus * item_cap, far.data(), sizeof(float4) * kClus,
                            cudaMemcpyHostToDevice) == cudaSuccess;
        }
        if (ok) ok = cudaMemset(c->sysred, 0, sizeof(double) * (size_t)S * kRed) == cudaSuccess;
        if (!ok) {
            free_ctx(c);
            return RBSOG_ENOMEM;
        }

        // ---- constants
        c->sc.M = P.M; c->sc.ME = P.M_energy; c->sc.rc = P.rc; c->sc.ke = P.ke;
        for (int l = 0; l < MM; ++l) {
            c->sc.w[l] = w[l]; c->sc.s[l] = s[l]; c->sc.wt[l] = wt[l]; c->sc.st[l] = st[l];
            c->sc.wf[l] = (float)w[l]; c->sc.wtf[l] = (float)wt[l];
            c->sc.is2f[l] = (float)(1.0 / (s[l] * s[l])); c->sc.ist2f[l] = (float)(1.0 / (st[l] * st[l]));
        }
        c->pcf.M = c->pcd.M = P.M;
        c->pcf.ME = c->pcd.ME = P.M_energy;
        c->pcf.rc2 = (float)(P.rc * P.rc); c->pcd.rc2 = P.rc * P.rc; c->pcf.rc2d = P.rc * P.rc;
        c->pcf.rc2_hi = (float)(P.rc * P.rc * (1.0 + 1e-5));
        c->pcf.rc2_lo = (float)(P.rc * P.rc * (1.0 - 1e-5));
        c->pcf.rl2_hi = (float)(list_radius(P) * list_radius(P) * (1.0 + 1e-5));
        c->pcf.ke = (float)P.ke; c->pcd.ke = P.ke;
        for (int l = 0; l < MM; ++l) {
            c->pcd.inv_s2[l] = 1.0 / (s[l] * s[l]);
            c->pcd.w[l] = w[l];
            c->pcd.wt[l] = l < P.M ? wt[l] : 0.0;
        }
        {
            // FP64 split: Gaussians with s_l >= 0.8 r_c go into a Taylor tail in u = r^2
            const double swide = 0.8 * P.rc;
            int nf = 0;
            while (nf < MM && s[nf] < swide && st[nf] < swide) ++nf;
            c->pcd.nf = nf;
            c->pcd.rc2f = (float)(P.rc * P.rc * (1.0 + 1e-5));
            for (int k = 0; k <= kTailD; ++k) {
                double tk = 0.0, ek = 0.0, fact = 1.0;
                for (int i = 2; i <= k; ++i) fact *= i;
                for (int l = nf; l < P.M; ++l) tk += wt[l] * std::pow(-1.0 / (st[l] * st[l]), k) / fact;
                for (int l = nf; l < P.M_energy; ++l) ek += w[l] * std::pow(-1.0 / (s[l] * s[l]), k) / fact;
                c->pcd.tt[k] = tk;
                c->pcd.te[k] = ek;
            }
        }
        {
            // FP32 split: Taylor tails in u = r^2 for the force Gaussians with
            // s~_l >= 1.3 r_c and the energy Gaussians with s_l >= 2.5 r_c
            const double swide = 2.5 * P.rc, swide_f = 1.3 * P.rc, log2e = 1.4426950408889634;
            int nff = 0, nfe = 0;
            while (nff < P.M && st[nff] < swide_f) ++nff;
            while (nfe < P.M_energy && s[nfe] < swide) ++nfe;
            c->pcf.nff = nff;
            c->pcf.nfe = nfe;
            for (int l = 0; l < MM; ++l) {
                c->pcf.beta[l] = (float)(log2e / (st[l] * st[l]));
                c->pcf.wt[l] = l < P.M ? (float)wt[l] : 0.f;
                const double be = log2e / (s[l] * s[l]);
                c->pcf.be_hi[l] = (float)be;
                c->pcf.be_lo[l] = (float)(be - (double)c->pcf.be_hi[l]);
                c->pcf.w_hi[l] = (float)w[l];
                c->pcf.w_lo[l] = (float)(w[l] - (double)c->pcf.w_hi[l]);
            }
            // force tail sum_{l >= nff} w~_l e^{-u/s~_l^2} on u in [0, r_c^2 (1 + 1e-5)]:
            // the polynomial of degree kTailF through its values at the kTailF + 1
            // Chebyshev nodes of the interval (within 1e-8 of the tail's value at
            // u = 0 for Table 2 row 2, below the FP32 rounding of its evaluation)
            {
                const int D = kTailF;
                const double U = P.rc * P.rc * (1.0 + 1e-5);
                double A[kTailF + 1][kTailF + 2];
                for (int k = 0; k <= D; ++k) {
                    const double t = 0.5 * (1.0 - std::cos((2 * k + 1) * kPi / (2.0 * (D + 1))));   // node / U
                    double tv = 0.0;
                    for (int l = nff; l < P.M; ++l) tv += wt[l] * std::exp(-(t * U) / (st[l] * st[l]));
                    double pw = 1.0;
                    for (int j = 0; j <= D; ++j) { A[k][j] = pw; pw *= t; }
                    A[k][D + 1] = tv;
                }
                // Gaussian elimination with partial pivoting (in t = u / U)
                for (int col = 0; col <= D; ++col) {
                    int piv = col;
                    for (int r2 = col + 1; r2 <= D; ++r2)
                        if (std::fabs(A[r2][col]) > std::fabs(A[piv][col])) piv = r2;
                    for (int j = 0; j <= D + 1; ++j) std::swap(A[col][j], A[piv][j]);
                    for (int r2 = col + 1; r2 <= D; ++r2) {
                        const double f = A[r2][col] / A[col][col];
                        for (int j = col; j <= D + 1; ++j) A[r2][j] -= f * A[col][j];
                    }
                }
                double a[kTailF + 1];
                for (int k = D; k >= 0; --k) {
                    double v = A[k][D + 1];
                    for (int j = k + 1; j <= D; ++j) v -= A[k][j] * a[j];
                    a[k] = v / A[k][k];
                }
                double scale = 1.0;
                for (int k = 0; k <= D; ++k) { c->pcf.tt[k] = (float)(a[k] / scale); scale *= U; }
            }
            double te0 = 0.0;
            for (int k = 0; k <= kTail; ++k) {
                double ek = 0.0, fact = 1.0;
                for (int i = 2; i <= k; ++i) fact *= i;
                for (int l = nfe; l < P.M_energy; ++l) ek += w[l] * std::pow(-1.0 / (s[l] * s[l]), k) / fact;
                c->pcf.te[k] = k == 0 ? 0.f : (float)ek;
                if (k == 0) te0 = ek;
            }
            c->pcf.te0 = te0;
        }
        // LJ: one ntypes x ntypes block per system (uploaded with the buffers above)
        fill_sampler_args(P, wt, st, c->sa);
        c->ia.dt = P.dt; c->ia.T = P.T; c->ia.Pext = P.P_ext; c->ia.gamma = P.gamma; c->ia.gamma_box = P.gamma_box;
        c->ia.kB = kKB; c->ia.ftm2v = kFtm2v; c->ia.nktv2p = kNktv2p; c->ia.seed = P.seed; 
        c->ia.c_atom = std::exp(-P.gamma * P.dt);
        c->ia.c_box = std::exp(-P.gamma_box * P.dt);
        c->ia.ke = P.ke;
        c->ia.inv_m = c->inv_m; c->ia.sdv = c->sdv;
        c->ia.noise_f32 = P.precision == RBSOG_FP32 ? 1 : 0;

        c->b.S = S; c->b.N = N; c->b.C = C; c->b.sub = P.cell_sub; c->b.rc = P.rc; c->b.sys = c->sys;
        c->b.rlist = list_radius(P);
        c->b.skin = c->b.rlist > P.rc ? 1 : 0;
        c->b.atom_sys = c->atom_sys; c->b.cell_sys = c->cell_sys; c->b.item_sys = c->item_sys; c->b.chunk_sys = c->chunk_sys;
        c->b.chunk_a0 = c->chunk_a0; c->b.chunk_n = c->chunk_n; c->b.nchunks = c->nchunks;
        c->b.item_cap = item_cap;
        c->a.r = c->r; c->a.p = c->p; c->a.F = c->F; c->a.q = c->q; c->a.mass = c->mass; c->a.type = c->type;
        c->a.mol = c->mol; c->a.cell = c->cell; c->a.rank = c->rank; c->a.locf = c->locf; c->a.locd = c->locd;
        c->a.su = c->su; c->a.xref = c->xref; c->a.count = c->count; c->a.start = c->start; c->a.sidx = c->sidx; c->a.pos4 = c->pos4;
        c->a.qt = c->qt; c->a.posd = c->posd; c->a.aux = c->aux; c->a.items = c->items;
        c->a.posf = c->posf; c->a.ffix = c->ffix; c->a.ccl = c->ccl; c->a.cbox = c->cbox;
        c->a.ljd = c->ljd; c->a.ljf = c->ljf; c->a.ljf_lo = c->ljf_lo; c->a.turn_tab_d = c->turn_tab_d;
        c->m.nmol = nmolx; c->m.b_start = c->b_start; c->m.a_start = c->a_start; c->m.e_start = c->e_start;
        c->m.bonds = c->bonds; c->m.bk = c->bk; c->m.br0 = c->br0; c->m.angles = c->angles; c->m.ak = c->ak;
        c->m.at0 = c->at0; c->m.excl = c->excl; c->m.mchunk_sys = c->mchunk_sys; c->m.mchunk_m0 = c->mchunk_m0;
        c->m.mchunk_n = c->mchunk_n; c->m.nmchunks = c->nmchunks;

        e = prepare_sampler(P.P);
        if (e == cudaSuccess) e = prepare_pair();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { rbsog_status rr = cuda_fail(c, e, "create"); free_ctx(c); return rr; }
        // tilted cells: the sampler's lattice sums, once (the cell is held fixed)
        c->h_tilt.assign(3 * (size_t)S, 0.0);
        if (any_tri) {
            std::vector<SampScratch> hss(S);
            std::memset(hss.data(), 0, sizeof(SampScratch) * S);
            std::vector<int> tri_sys;
            int mmx[3] = {0, 0, 0};
            size_t tab = 0;
            for (int k = 0; k < S; ++k) {
                for (int a = 0; a < 3; ++a) c->h_tilt[3 * k + a] = systems[k].tilt[a];
                if (!tilted(systems[k])) continue;
                int mm[3];
                tri_range(systems[k].box, systems[k].tilt, st[0], mm);
                for (int a = 0; a < 3; ++a) { hss[k].tmm[a] = mm[a]; mmx[a] = std::max(mmx[a], mm[a]); }
                hss[k].tab0 = (long long)tab;
                tab += tri_tab_size(P.M, mm);
                tri_sys.push_back(k);
            }
            int *d_tri = nullptr;
            bool ok2 = dalloc(c, c->tri_tab, tab) && dalloc(c, d_tri, tri_sys.size()) &&
                       cudaMemcpy(c->samp, hss.data(), sizeof(SampScratch) * S, cudaMemcpyHostToDevice) == cudaSuccess &&
                       cudaMemcpy(d_tri, tri_sys.data(), sizeof(int) * tri_sys.size(), cudaMemcpyHostToDevice) == cudaSuccess;
            if (!ok2) { free_ctx(c); return RBSOG_ENOMEM; }
            c->sa.tri_tab = c->tri_tab;
            c->sa.has_tri = 1;
            launch_tri_tables(c->b, c->sa, c->samp, d_tri, (int)tri_sys.size(), mmx, c->st);
            e = cudaStreamSynchronize(c->st);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) { rbsog_status rr = cuda_fail(c, e, "tilted-cell tables"); free_ctx(c); return rr; }
        }
        // the first evaluation (counter 0) primes forces, virial and kinetic tensor
        launch_clear_flags(c->b, c->st);
        enqueue_eval(c, 0, 0, 1, 0);
        c->h_step = 0;
        e = cudaStreamSynchronize(c->st);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) { rbsog_status rr = cuda_fail(c, e, "first evaluation"); free_ctx(c); return rr; }
        rbsog_status fs = check_flags(c);
        if (fs != RBSOG_OK) { free_ctx(c); return fs; }
    } catch (const std::exception &ex) {
        free_ctx(c);
        return RBSOG_ENOMEM;
    }
    *out = c;
    return RBSOG_OK;
}

}  // namespace

extern "C" {

rbsog_status rbsog_create(const rbsog_params *params, int n_systems, const rbsog_system_desc *systems,
                          void *stream, rbsog_ctx **out)
{
    if (!systems) return RBSOG_EINVAL;
    return create_impl(params, n_systems, systems, nullptr, stream, out);
}

rbsog_status rbsog_pool_create(const rbsog_params *params, int n_slots, const rbsog_slot_caps *caps, void *stream,
                               rbsog_ctx **out)
{
    if (!caps || n_slots <= 0) return RBSOG_EINVAL;
    std::vector<SlotCaps> sc(n_slots);
    for (int k = 0; k < n_slots; ++k) {
        const rbsog_slot_caps &c = caps[k];
        if (c.max_atoms < 1 || c.max_molecules < 1 || c.max_molecules > c.max_atoms || c.max_bonds < 0 ||
            c.max_angles < 0 || c.max_excl < 0 || c.max_types < 1 || c.max_types > kMaxTypes)
            return RBSOG_EINVAL;
        sc[k].atoms = c.max_atoms; sc[k].mols = c.max_molecules; sc[k].bonds = c.max_bonds;
        sc[k].angles = c.max_angles; sc[k].excl = c.max_excl; sc[k].types = c.max_types;
        if (!(c.max_density > 0)) return RBSOG_EINVAL;
        sc[k].rho = c.max_density;
        for (int a = 0; a < 3; ++a) {
            if (!(c.max_box[a] > 0)) return RBSOG_EBOX;
            sc[k].box[a] = c.max_box[a];
        }
    }
    return create_impl(params, n_slots, nullptr, sc.data(), stream, out);
}

rbsog_status rbsog_pool_load(rbsog_ctx *c, int slot, const rbsog_system_desc *sys, int nsteps)
{
    if (!c || !c->pool || slot < 0 || slot >= c->S || !sys || nsteps == 0 || nsteps < -1) return RBSOG_EINVAL;
    rbsog_status vs = validate_system(*sys);
    if (vs != RBSOG_OK) return fail(c, vs, "rbsog_pool_load: invalid system");
    if (tilted(*sys)) return fail(c, RBSOG_EUNSUPPORTED, "rbsog_pool_load: tilted cells are served by rbsog_create contexts");
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pool load");
    DevSys ds;
    e = cudaMemcpy(&ds, c->sys + slot, sizeof(DevSys), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "pool load");
    if (ds.n != 0) return fail(c, RBSOG_EINVAL, "rbsog_pool_load: slot " + std::to_string(slot) + " is not empty");
    const SlotLayout &ly = c->lay[slot];
    SlotImage im;
    std::string why;
    if (!build_image(c->prm, ly, ds, *sys, c->sog_w, im, why))
        return fail(c, RBSOG_EINVAL, "rbsog_pool_load: slot " + std::to_string(slot) + ": " + why);
    ds.act = 1;
    ds.steps_left = nsteps;
    ds.list_valid = 0;
    ds.list_builds = 0;
    c->slot_err[slot] = RBSOG_OK;
    auto put = [&](auto *dst, const auto &v) {
        if (e == cudaSuccess && !v.empty())
            e = cudaMemcpy(dst, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice);
    };
    const size_t A0 = ly.atom0;
    put(c->r + 3 * A0, im.r); put(c->p + 3 * A0, im.p); put(c->q + A0, im.q); put(c->mass + A0, im.mass);
    put(c->inv_m + A0, im.inv_m); put(c->sdv + A0, im.sdv); put(c->type + A0, im.type); put(c->mol + A0, im.mol);
    put(c->b_start + ly.mol0, im.b_start); put(c->a_start + ly.mol0, im.a_start); put(c->e_start + ly.mol0, im.e_start);
    put(c->bonds + 2 * (size_t)ly.bond0, im.bonds); put(c->bk + ly.bond0, im.bk); put(c->br0 + ly.bond0, im.br0);
    put(c->angles + 3 * (size_t)ly.angle0, im.angles); put(c->ak + ly.angle0, im.ak); put(c->at0 + ly.angle0, im.at0);
    put(c->excl + 2 * (size_t)ly.excl0, im.excl);
    put(c->ljd + ly.lj0, im.ljd); put(c->ljf + ly.lj0, im.ljf); put(c->ljf_lo + ly.lj0, im.ljf_lo);
    if (e == cudaSuccess) e = cudaMemcpy(c->self_e + 2 * slot, im.self_e, 2 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->sys + slot, &ds, sizeof(DevSys), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "pool load");
    c->h_n[slot] = sys->n_atoms;
    return RBSOG_OK;
}

rbsog_status rbsog_pool_prime(rbsog_ctx *c)
{
    if (!c) return RBSOG_EINVAL;
    launch_clear_flags(c->b, c->st);
    enqueue_eval(c, 0, 0, 1, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "pool prime");
    return check_flags(c);
}

rbsog_status rbsog_pool_state(rbsog_ctx *c, int *state, unsigned long long *step, int *err)
{
    if (!c || !state) return RBSOG_EINVAL;
    std::vector<DevSys> h(c->S);
    cudaError_t e = cudaMemcpyAsync(h.data(), c->sys, sizeof(DevSys) * c->S, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pool state");
    for (int s = 0; s < c->S; ++s) {
        const bool failed = c->pool && c->slot_err[s] != RBSOG_OK;
        state[s] = h[s].n == 0 ? 0 : (h[s].act ? 1 : (failed ? 3 : 2));
        if (step) step[s] = h[s].step;
        if (err) err[s] = c->pool ? (int)c->slot_err[s] : 0;
    }
    return RBSOG_OK;
}

rbsog_status rbsog_pool_unload(rbsog_ctx *c, int slot, double *r, double *v, rbsog_result *res)
{
    if (!c || !c->pool || slot < 0 || slot >= c->S) return RBSOG_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->st);
    DevSys ds;
    if (e == cudaSuccess) e = cudaMemcpy(&ds, c->sys + slot, sizeof(DevSys), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "pool unload");
    if (ds.n == 0) return fail(c, RBSOG_EINVAL, "rbsog_pool_unload: slot " + std::to_string(slot) + " is empty");
    const size_t A0 = c->lay[slot].atom0, n = ds.n;
    if (r) e = cudaMemcpy(r, c->r + 3 * A0, 3 * n * sizeof(double), cudaMemcpyDeviceToHost);
    if (v && e == cudaSuccess) {
        std::vector<double> p(3 * n), m(n);
        e = cudaMemcpy(p.data(), c->p + 3 * A0, 3 * n * sizeof(double), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(m.data(), c->mass + A0, n * sizeof(double), cudaMemcpyDeviceToHost);
        for (size_t i = 0; e == cudaSuccess && i < 3 * n; ++i) v[i] = p[i] / m[i / 3];
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "pool unload");
    if (res) {
        std::vector<rbsog_result> all(c->S);
        rbsog_status fs = fill_results(c, all.data());
        if (fs != RBSOG_OK) return fs;
        *res = all[slot];
    }
    ds.n = 0; ds.nmol = 0; ds.act = 0; ds.steps_left = 0; ds.flags = 0; ds.nD = 0;
    e = cudaMemcpy(c->sys + slot, &ds, sizeof(DevSys), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "pool unload");
    c->h_n[slot] = 0;
    return RBSOG_OK;
}

rbsog_status rbsog_set_box(rbsog_ctx *c, int s, const double box[3], int rescale)
{
    if (!c || s < 0 || s >= c->S || !box) return RBSOG_EINVAL;
    if (!c->h_tilt.empty() && (c->h_tilt[3 * s] != 0.0 || c->h_tilt[3 * s + 1] != 0.0 || c->h_tilt[3 * s + 2] != 0.0))
        return fail(c, RBSOG_EUNSUPPORTED, "set_box: a tilted cell is held fixed");
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 0) || (int)std::floor(box[a] * c->prm.cell_sub / list_radius(c->prm)) < 2 * c->prm.cell_sub + 1)
            return fail(c, RBSOG_EBOX, "box edge below 3 cells");
    DevSys h;
    cudaError_t e = cudaMemcpyAsync(&h, c->sys + s, sizeof(DevSys), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_box");
    if (rescale) {
        std::vector<double> r(3 * (size_t)c->h_n[s]);
        double *dr = c->r + 3 * (size_t)c->h_atom0[s];
        e = cudaMemcpy(r.data(), dr, r.size() * sizeof(double), cudaMemcpyDeviceToHost);
        for (size_t i = 0; i < r.size(); ++i) r[i] *= box[i % 3] / h.L[i % 3];
        if (e == cudaSuccess) e = cudaMemcpy(dr, r.data(), r.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(c, e, "set_box");
    }
    for (int a = 0; a < 3; ++a) h.L[a] = box[a];
    h.V = box[0] * box[1] * box[2];
    h.list_valid = 0;
    e = cudaMemcpy(c->sys + s, &h, sizeof(DevSys), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_box");
    return RBSOG_OK;
}

rbsog_status rbsog_set_positions(rbsog_ctx *c, const double *r, int on_device)
{
    if (!c || !r) return RBSOG_EINVAL;
    cudaError_t e = cudaMemcpyAsync(c->r, r, 3 * sizeof(double) * c->N,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_positions");
    launch_invalidate_lists(c->b, c->st);
    return RBSOG_OK;
}

rbsog_status rbsog_get_positions(rbsog_ctx *c, double *r, int on_device)
{
    if (!c || !r) return RBSOG_EINVAL;
    cudaError_t e = cudaMemcpyAsync(r, c->r, 3 * sizeof(double) * c->N,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_positions");
    return RBSOG_OK;
}

rbsog_status rbsog_get_velocities(rbsog_ctx *c, double *v, int on_device)
{
    if (!c || !v || on_device) return RBSOG_EINVAL;
    std::vector<double> p(3 * (size_t)c->N), m(c->N);
    cudaError_t e = cudaMemcpyAsync(p.data(), c->p, p.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m.data(), c->mass, m.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_velocities");
    for (size_t i = 0; i < p.size(); ++i) v[i] = p[i] / m[i / 3];
    return RBSOG_OK;
}

// The evaluation of rbsog_step as a CUDA graph (captured on first use; the
// step counter is set by a kernel launched before it).
static rbsog_status ensure_eval_graph(rbsog_ctx *c, int energy)
{
    if (c->eval_graph[energy]) return RBSOG_OK;
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "capture");
    launch_clear_flags(c->b, c->st);
    enqueue_eval(c, 0, 0, energy, 0);
    e = cudaStreamEndCapture(c->st, &g);
    if (e != cudaSuccess) return cuda_fail(c, e, "capture end");
    e = cudaGraphInstantiate(&c->eval_graph[energy], g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(c, e, "graph instantiate"); }
    c->eval_graph_src[energy] = g;
    return RBSOG_OK;
}

// Flags and (optionally) the per-system reductions of the last evaluation in
// one read-back: the two copies are enqueued, then the stream is waited for once.
static rbsog_status read_back(rbsog_ctx *c, std::vector<double> *red)
{
    std::vector<DevSys> h(c->S);
    cudaError_t e = cudaMemcpyAsync(h.data(), c->sys, sizeof(DevSys) * c->S, cudaMemcpyDeviceToHost, c->st);
    if (red && e == cudaSuccess) {
        red->resize((size_t)c->S * kRed);
        e = cudaMemcpyAsync(red->data(), c->sysred, red->size() * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "device");
    return process_flags(c, h);
}

rbsog_status rbsog_step(rbsog_ctx *c, uint64_t step, double *forces, int on_device, rbsog_result *res)
{
    if (!c) return RBSOG_EINVAL;
    launch_set_step(c->b, (unsigned long long)step, c->st);
    cudaError_t e = cudaSuccess;
    for (auto ev : c->t_events) cudaEventDestroy(ev);
    c->t_events.clear();
    c->t_names.clear();
    if (c->timing) {                          // eager, with events around each kernel
        launch_clear_flags(c->b, c->st);
        enqueue_eval(c, 0, 0, 1, 0);
    } else {
        rbsog_status gs = ensure_eval_graph(c, 1);
        if (gs != RBSOG_OK) return gs;
        e = cudaGraphLaunch(c->eval_graph[1], c->st);
        if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    }
    c->h_step = (unsigned long long)step;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
    if (forces) {
        e = cudaMemcpyAsync(forces, c->F, 3 * sizeof(double) * c->N,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st);
        if (e != cudaSuccess) return cuda_fail(c, e, "forces");
    }
    std::vector<double> red;
    rbsog_status fs = read_back(c, res ? &red : nullptr);
    if (fs != RBSOG_OK) return fs;
    if (c->timing) {
        c->t_ms.clear();
        for (size_t k = 1; k < c->t_events.size(); ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, c->t_events[k - 1], c->t_events[k]);
            c->t_ms.push_back(ms);
        }
    }
    if (res) results_from(c, red, res);
    return RBSOG_OK;
}

rbsog_status rbsog_step_forces(rbsog_ctx *c, uint64_t step, double *forces, int on_device, double *virial)
{
    if (!c) return RBSOG_EINVAL;
    launch_set_step(c->b, (unsigned long long)step, c->st);
    rbsog_status gs = ensure_eval_graph(c, 0);
    if (gs != RBSOG_OK) return gs;
    cudaError_t e = cudaGraphLaunch(c->eval_graph[0], c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    c->h_step = (unsigned long long)step;
    if (forces) {
        e = cudaMemcpyAsync(forces, c->F, 3 * sizeof(double) * c->N,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st);
        if (e != cudaSuccess) return cuda_fail(c, e, "forces");
    }
    std::vector<double> red;
    rbsog_status fs = read_back(c, virial ? &red : nullptr);
    if (fs != RBSOG_OK) return fs;
    if (virial)
        for (int s = 0; s < c->S; ++s)
            for (int k = 0; k < 9; ++k) virial[9 * s + k] = red[(size_t)s * kRed + 9 + kSym[k]];
    return RBSOG_OK;
}

static rbsog_status ensure_graph(rbsog_ctx *c, int energy)
{
    cudaError_t e;
    if (!c->graph[energy]) {
        bool t = c->timing;
        c->timing = false;
        cudaGraph_t g;
        e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(c, e, "capture");
        enqueue_npt_step(c, energy);
        e = cudaStreamEndCapture(c->st, &g);
        c->timing = t;
        if (e != cudaSuccess) return cuda_fail(c, e, "capture end");
        e = cudaGraphInstantiate(&c->graph[energy], g, 0);
        if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(c, e, "graph instantiate"); }
        c->graph_src[energy] = g;
        // the event-record nodes around the pair kernel
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev = nullptr;
            if (cudaGraphEventRecordNodeGetEvent(nd, &ev) != cudaSuccess) continue;
            for (int k = 0; k < 2; ++k)
                if (ev == c->ev_pair_ph[k]) c->pair_node[energy][k] = nd;
        }
    }
    return RBSOG_OK;
}

// Point the pair-kernel event nodes of graph `en` at the next ring entry (or
// back at the placeholders once the ring is used up).
static void arm_pair_trace(rbsog_ctx *c, int en)
{
    if (!c->pair_node[en][0] || !c->pair_node[en][1]) return;
    if (c->ring_pos < (int)c->ring_s.size()) {
        cudaGraphExecEventRecordNodeSetEvent(c->graph[en], c->pair_node[en][0], c->ring_s[c->ring_pos]);
        cudaGraphExecEventRecordNodeSetEvent(c->graph[en], c->pair_node[en][1], c->ring_e[c->ring_pos]);
        c->pair_node_live[en] = true;
        ++c->ring_pos;
    } else if (c->pair_node_live[en]) {
        cudaGraphExecEventRecordNodeSetEvent(c->graph[en], c->pair_node[en][0], c->ev_pair_ph[0]);
        cudaGraphExecEventRecordNodeSetEvent(c->graph[en], c->pair_node[en][1], c->ev_pair_ph[1]);
        c->pair_node_live[en] = false;
    }
}

// Enqueue nsteps graph steps; energies on steps whose counter is a multiple
// of thermo_every, and on the last one when last_energy is set.
static rbsog_status run_steps(rbsog_ctx *c, int nsteps, bool last_energy)
{
    if (!c || nsteps < 0) return RBSOG_EINVAL;
    if (c->prm.dt <= 0) return fail(c, RBSOG_EINVAL, "dt must be positive");
    for (int n = 0; n < nsteps; ++n) {
        const unsigned long long next = c->h_step + 1ull;
        const int en = (last_energy && n == nsteps - 1) ||
                       (c->prm.thermo_every > 0 && next % (unsigned long long)c->prm.thermo_every == 0);
        rbsog_status gs = ensure_graph(c, en);
        if (gs != RBSOG_OK) return gs;
        arm_pair_trace(c, en);
        cudaError_t e = cudaGraphLaunch(c->graph[en], c->st);
        if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
        c->h_step = next;
    }
    return RBSOG_OK;
}

rbsog_status rbsog_run_async(rbsog_ctx *c, int nsteps) { return run_steps(c, nsteps, false); }

rbsog_status rbsog_set_thermo_every(rbsog_ctx *c, int every)
{
    if (!c || every < 0) return RBSOG_EINVAL;
    c->prm.thermo_every = every;
    return RBSOG_OK;
}

rbsog_status rbsog_sync(rbsog_ctx *c)
{
    if (!c) return RBSOG_EINVAL;
    rbsog_status fs = check_flags(c);
    launch_clear_flags(c->b, c->st);
    return fs;
}

rbsog_status rbsog_sync_timeout(rbsog_ctx *c, double timeout_ms)
{
    if (!c || !(timeout_ms >= 0.0) || !std::isfinite(timeout_ms)) return RBSOG_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaStreamQuery(c->st);
        if (e == cudaSuccess) return rbsog_sync(c);
        if (e != cudaErrorNotReady) return cuda_fail(c, e, "sync");
        const double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (el >= timeout_ms)
            return fail(c, RBSOG_ETIMEOUT, "rbsog_sync_timeout: the enqueued steps still run after " +
                                               std::to_string(timeout_ms) + " ms");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

void *rbsog_stream(rbsog_ctx *c) { return c ? (void *)c->st : nullptr; }

rbsog_status rbsog_run(rbsog_ctx *c, int nsteps, rbsog_result *last)
{
    if (!c || nsteps < 0) return RBSOG_EINVAL;
    launch_clear_flags(c->b, c->st);
    rbsog_status rs = run_steps(c, nsteps, true);
    if (rs != RBSOG_OK) return rs;
    std::vector<double> red;
    rbsog_status fs = read_back(c, last ? &red : nullptr);
    if (fs != RBSOG_OK) return fs;
    if (last) results_from(c, red, last);
    return RBSOG_OK;
}

rbsog_status rbsog_get_state(rbsog_ctx *c, void *buf, size_t *len)
{
    if (!c || !len) return RBSOG_EINVAL;
    const size_t need = sizeof(uint64_t) * 2 + 6 * sizeof(double) * (size_t)c->N + sizeof(DevSys) * c->S +
                        3 * sizeof(double) * (size_t)c->N + sizeof(double) * (size_t)c->S * kRed;
    if (!buf) { *len = need; return RBSOG_OK; }
    if (*len < need) return RBSOG_EINVAL;
    // header: the host step counter (the per-system Philox counters are in DevSys)
    cudaError_t e = cudaStreamSynchronize(c->st);
    uint64_t hdr[2] = {(uint64_t)c->h_step, (uint64_t)c->N};
    char *o = static_cast<char *>(buf);
    std::memcpy(o, hdr, sizeof(hdr));
    o += sizeof(hdr);
    if (e == cudaSuccess) e = cudaMemcpy(o, c->r, 3 * sizeof(double) * c->N, cudaMemcpyDeviceToHost);
    o += 3 * sizeof(double) * c->N;
    if (e == cudaSuccess) e = cudaMemcpy(o, c->p, 3 * sizeof(double) * c->N, cudaMemcpyDeviceToHost);
    o += 3 * sizeof(double) * c->N;
    if (e == cudaSuccess) e = cudaMemcpy(o, c->F, 3 * sizeof(double) * c->N, cudaMemcpyDeviceToHost);
    o += 3 * sizeof(double) * c->N;
    if (e == cudaSuccess) e = cudaMemcpy(o, c->sys, sizeof(DevSys) * c->S, cudaMemcpyDeviceToHost);
    o += sizeof(DevSys) * c->S;
    if (e == cudaSuccess) e = cudaMemcpy(o, c->sysred, sizeof(double) * c->S * kRed, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_state");
    *len = need;
    return RBSOG_OK;
}

rbsog_status rbsog_set_state(rbsog_ctx *c, const void *buf, size_t len)
{
    if (!c || !buf) return RBSOG_EINVAL;
    size_t need = 0;
    rbsog_get_state(c, nullptr, &need);
    if (len < need) return RBSOG_EINVAL;
    const uint64_t *h = static_cast<const uint64_t *>(buf);
    if (h[1] != (uint64_t)c->N) return fail(c, RBSOG_EINVAL, "state of another system size");
    unsigned long long step = h[0];
    const char *o = static_cast<const char *>(buf) + 2 * sizeof(uint64_t);
    cudaError_t e = cudaMemcpy(c->r, o, 3 * sizeof(double) * c->N, cudaMemcpyHostToDevice);
    o += 3 * sizeof(double) * c->N;
    if (e == cudaSuccess) e = cudaMemcpy(c->p, o, 3 * sizeof(double) * c->N, cudaMemcpyHostToDevice);
    o += 3 * sizeof(double) * c->N;
    if (e == cudaSuccess) e = cudaMemcpy(c->F, o, 3 * sizeof(double) * c->N, cudaMemcpyHostToDevice);
    o += 3 * sizeof(double) * c->N;
    if (e == cudaSuccess) e = cudaMemcpy(c->sys, o, sizeof(DevSys) * c->S, cudaMemcpyHostToDevice);
    o += sizeof(DevSys) * c->S;
    if (e == cudaSuccess) e = cudaMemcpy(c->sysred, o, sizeof(double) * c->S * kRed, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_state");
    launch_invalidate_lists(c->b, c->st);     // the lists are not part of the state
    c->h_step = step;
    return RBSOG_OK;
}

rbsog_status rbsog_debug_cells(rbsog_ctx *c, int s, int *ncell, int *cell_of_atom)
{
    if (!c || s < 0 || s >= c->S) return RBSOG_EINVAL;
    DevSys h;
    cudaError_t e = cudaMemcpy(&h, c->sys + s, sizeof(DevSys), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "debug_cells");
    if (ncell) for (int a = 0; a < 3; ++a) ncell[a] = h.ncell[a];
    if (cell_of_atom) {
        e = cudaMemcpy(cell_of_atom, c->cell + c->h_atom0[s], sizeof(int) * c->h_n[s], cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "debug_cells");
        for (int i = 0; i < c->h_n[s]; ++i) cell_of_atom[i] -= h.cell0;
    }
    return RBSOG_OK;
}

rbsog_status rbsog_debug_modes(rbsog_ctx *c, int s, int *mr, int *mnr, int *D, int *cr, int *cnr, int *nD,
                               double *S2, double *rho)
{
    if (!c || s < 0 || s >= c->S) return RBSOG_EINVAL;
    DevSys h;
    cudaError_t e = cudaMemcpy(&h, c->sys + s, sizeof(DevSys), cudaMemcpyDeviceToHost);
    const int P = c->prm.P, Dc = c->Dcap;
    if (e == cudaSuccess && mr) e = cudaMemcpy(mr, c->mr + (size_t)s * P * 3, sizeof(int) * P * 3, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && mnr) e = cudaMemcpy(mnr, c->mnr + (size_t)s * P * 3, sizeof(int) * P * 3, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && D) e = cudaMemcpy(D, c->D + (size_t)s * Dc * 3, sizeof(int) * 3 * h.nD, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && cr) e = cudaMemcpy(cr, c->cr + (size_t)s * Dc, sizeof(int) * h.nD, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && cnr) e = cudaMemcpy(cnr, c->cnr + (size_t)s * Dc, sizeof(int) * h.nD, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && rho) e = cudaMemcpy(rho, c->rho + (size_t)s * Dc * 2, sizeof(double) * 2 * h.nD, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "debug_modes");
    if (nD) *nD = h.nD;
    if (S2) { S2[0] = h.Sr; S2[1] = h.Snr; }
    return RBSOG_OK;
}

rbsog_status rbsog_virial_nr_shared(rbsog_ctx *c, double *out)
{
    if (!c || !out) return RBSOG_EINVAL;
    launch_nr_shared(c->b, c->D, c->cr, c->rho, c->Dcap, c->prm.P, c->prm.ke, c->sa, c->nrsh, c->st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, c->nrsh, sizeof(double) * 9 * (size_t)c->S, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "virial_nr_shared");
    return RBSOG_OK;
}

rbsog_status rbsog_set_timing(rbsog_ctx *c, int enable)
{
    if (!c) return RBSOG_EINVAL;
    c->timing = enable != 0;
    return RBSOG_OK;
}

rbsog_status rbsog_get_timing(rbsog_ctx *c, int max, char *names, double *ms, int *count)
{
    if (!c || !count) return RBSOG_EINVAL;
    int n = std::min<int>(max, (int)c->t_ms.size());
    for (int k = 0; k < n; ++k) {
        if (ms) ms[k] = c->t_ms[k];
        if (names) {
            std::strncpy(names + 32 * k, c->t_names[k + 1].c_str(), 31);
            names[32 * k + 31] = 0;
        }
    }
    *count = n;
    return RBSOG_OK;
}

rbsog_status rbsog_trace_pair(rbsog_ctx *c, int nsteps)
{
    if (!c || nsteps < 0) return RBSOG_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "trace");
    // point every graph node back at the placeholders before the ring's events go
    for (int en = 0; en < 2; ++en) {
        if (!c->pair_node_live[en]) continue;
        cudaGraphExecEventRecordNodeSetEvent(c->graph[en], c->pair_node[en][0], c->ev_pair_ph[0]);
        cudaGraphExecEventRecordNodeSetEvent(c->graph[en], c->pair_node[en][1], c->ev_pair_ph[1]);
        c->pair_node_live[en] = false;
    }
    for (auto ev : c->ring_s) cudaEventDestroy(ev);
    for (auto ev : c->ring_e) cudaEventDestroy(ev);
    c->ring_s.assign(nsteps, nullptr);
    c->ring_e.assign(nsteps, nullptr);
    for (int k = 0; k < nsteps; ++k) {
        e = cudaEventCreate(&c->ring_s[k]);
        if (e == cudaSuccess) e = cudaEventCreate(&c->ring_e[k]);
        if (e != cudaSuccess) return cuda_fail(c, e, "trace events");
    }
    c->ring_pos = 0;
    return RBSOG_OK;
}

rbsog_status rbsog_trace_pair_times(rbsog_ctx *c, int max, double *ms, int *count)
{
    if (!c || !count) return RBSOG_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "trace");
    const int n = std::min(max, c->ring_pos);
    for (int k = 0; k < n; ++k) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, c->ring_s[k], c->ring_e[k]);
        if (e != cudaSuccess) return cuda_fail(c, e, "trace times");
        if (ms) ms[k] = t;
    }
    *count = n;
    return RBSOG_OK;
}

size_t rbsog_structure_factor_workspace(int n_atoms, int nD)
{
    if (n_atoms < 1 || nD < 1) return 0;
    return sk_stateless_workspace(n_atoms, nD);
}

rbsog_status rbsog_structure_factor(const double *r, const double *q, int n_atoms, const double box[3],
                                    const int *m, int nD, double *rho, void *work, int precision, void *stream)
{
    if (!r || !q || !box || !m || !rho || !work || n_atoms < 1 || nD < 1 || (precision != 0 && precision != 1))
        return RBSOG_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 0)) return RBSOG_EBOX;
    cudaError_t e = sk_stateless(r, q, n_atoms, box, m, nD, rho, work, precision, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RBSOG_OK : RBSOG_ECUDA;
}

rbsog_status rbsog_structure_factor_noalloc(const double *r, const double *q, int n_atoms, const double box[3],
                                            const int *m, int nD, double *rho, int precision, void *stream)
{
    if (!r || !q || !box || !m || !rho || n_atoms < 1 || nD < 1 || (precision != 0 && precision != 1))
        return RBSOG_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 0)) return RBSOG_EBOX;
    const size_t need = sk_stateless_workspace(n_atoms, nD);
    if (need > kSkStaticBytes) {
        g_create_err = "rbsog_structure_factor_noalloc: " + std::to_string(n_atoms) + " atoms and " +
                       std::to_string(nD) + " modes need " + std::to_string(need) +
                       " bytes of scratch; the fixed scratch holds " + std::to_string(kSkStaticBytes);
        return RBSOG_EOVERFLOW;
    }
    void *work = nullptr;
    cudaError_t e = sk_static_scratch(&work);
    if (e != cudaSuccess) {
        g_create_err = std::string("rbsog_structure_factor_noalloc: scratch set-up: ") + cudaGetErrorString(e);
        return RBSOG_ECUDA;
    }
    e = sk_stateless(r, q, n_atoms, box, m, nD, rho, work, precision, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RBSOG_OK : RBSOG_ECUDA;
}

rbsog_status rbsog_autotune(const rbsog_params *params, int n_systems, const rbsog_system_desc *systems,
                            int nsteps, void *stream, rbsog_params *best, double *times)
{
    if (!params || !systems || n_systems < 1 || !best || nsteps < 1) return RBSOG_EINVAL;
    rbsog_status vs = validate_params(params);
    if (vs != RBSOG_OK) return vs;
    const bool f32 = params->precision == RBSOG_FP32;
    const int ncols = f32 ? 4 : 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best_ms = 1e300;
    int k = 0;
    for (int sub = 1; sub <= 2; ++sub) {
        for (int col = 1; col <= ncols; ++col, ++k) {
            rbsog_params p = *params;
            p.cell_sub = sub;
            p.cluster_cols = f32 ? col : 0;
            if (times) times[k] = -1.0;
            rbsog_ctx *c = nullptr;
            if (rbsog_create(&p, n_systems, systems, stream, &c) != RBSOG_OK) continue;   // box too small for the cells
            std::vector<double> ms;
            bool ok = rbsog_run(c, 3, nullptr) == RBSOG_OK;   // warm-up (and the step graphs)
            for (int t = 0; ok && t < nsteps; ++t) {
                cudaEventRecord(e0, c->st);
                ok = rbsog_run_async(c, 1) == RBSOG_OK;
                cudaEventRecord(e1, c->st);
                float m = 0.f;
                if (ok) ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&m, e0, e1) == cudaSuccess;
                ms.push_back(m);
            }
            if (ok) ok = rbsog_sync(c) == RBSOG_OK;
            rbsog_destroy(c);
            if (!ok || ms.empty()) continue;
            std::sort(ms.begin(), ms.end());
            const double med = ms[ms.size() / 2];
            if (times) times[k] = med;
            if (med < best_ms) {
                best_ms = med;
                *best = p;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!(best_ms < 1e300)) return fail(nullptr, RBSOG_EINVAL, "rbsog_autotune: no candidate shape runs");
    return RBSOG_OK;
}

int rbsog_modes_capacity(const rbsog_params *p)
{
    if (!p || p->P < 1) return 0;
    return p->sampler == RBSOG_SAMPLER_IID ? 2 * p->P : p->P + 1;
}

rbsog_status rbsog_modes(const rbsog_params *params, const double box[3], uint64_t rng_id, uint64_t step, int *D,
                         int *cr, int *cnr, int *nD, double *S, void *stream)
{
    if (!params || !box || !D || !cr || !cnr || !nD) return fail(nullptr, RBSOG_EINVAL, "rbsog_modes: null argument");
    rbsog_status vs = validate_params(params);
    if (vs != RBSOG_OK) return fail(nullptr, vs, "rbsog_modes: bad parameters");
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 0) || !std::isfinite(box[a])) return fail(nullptr, RBSOG_EBOX, "rbsog_modes: box edge <= 0");
    const rbsog_params &P = *params;
    std::vector<double> w, s, wt, st;
    sog_terms(P, P.M, w, s, wt, st);
    SamplerArgs sa{};
    fill_sampler_args(P, wt, st, sa);
    const int Pn = P.P, Dcap = rbsog_modes_capacity(params);
    // one system of one atom (the sampler reads only its box, key and counter)
    DevSys h;
    std::memset(&h, 0, sizeof(h));
    for (int a = 0; a < 3; ++a) h.L[a] = box[a];
    h.V = box[0] * box[1] * box[2];
    h.act = 1;
    h.n = 1;
    h.rng_id = rng_id;
    h.step = step;
    const size_t nb_sys = ((sizeof(DevSys) + 255) / 256) * 256, nb_ss = ((sizeof(SampScratch) + 255) / 256) * 256;
    const size_t nb_i = (size_t)(2 * 3 * Pn + 3 * Dcap + 2 * Dcap) * sizeof(int);
    const size_t nb_pm = (size_t)Pn * sizeof(int4), nb_d = (size_t)4 * Pn * sizeof(double);
    const size_t total = nb_sys + nb_ss + ((nb_i + 255) / 256) * 256 + ((nb_pm + 255) / 256) * 256 + nb_d;
    char *buf = nullptr;
    ++g_dev_alloc_calls;
    cudaError_t e = cudaMalloc(&buf, total);
    if (e != cudaSuccess) return fail(nullptr, RBSOG_ENOMEM, "rbsog_modes: device memory");
    DevSys *dsys = reinterpret_cast<DevSys *>(buf);
    SampScratch *ss = reinterpret_cast<SampScratch *>(buf + nb_sys);
    int *ib = reinterpret_cast<int *>(buf + nb_sys + nb_ss);
    int *mr = ib, *mnr = ib + 3 * Pn, *dD = ib + 6 * Pn, *dcr = dD + 3 * Dcap, *dcnr = dcr + Dcap;
    int4 *pm = reinterpret_cast<int4 *>(buf + nb_sys + nb_ss + ((nb_i + 255) / 256) * 256);
    double *pd = reinterpret_cast<double *>(reinterpret_cast<char *>(pm) + ((nb_pm + 255) / 256) * 256);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    e = prepare_sampler(Pn);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dsys, &h, sizeof(h), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) {
        Batch b{};
        b.S = 1;
        b.sys = dsys;
        launch_sampler(b, sa, 0, mr, mnr, dD, dcr, dcnr, pm, pd, pd + Pn, pd + 2 * Pn, pd + 3 * Pn, ss, Dcap, cs);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, dsys, sizeof(h), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e == cudaSuccess && h.nD > 0) {
        e = cudaMemcpy(D, dD, sizeof(int) * 3 * h.nD, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(cr, dcr, sizeof(int) * h.nD, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(cnr, dcnr, sizeof(int) * h.nD, cudaMemcpyDeviceToHost);
    }
    ++g_dev_alloc_calls;
    cudaFree(buf);
    if (e != cudaSuccess) return fail(nullptr, RBSOG_ECUDA, std::string("rbsog_modes: ") + cudaGetErrorString(e));
    *nD = h.nD;
    if (S) { S[0] = h.Sr; S[1] = h.Snr; }
    return RBSOG_OK;
}

size_t rbsog_longrange_force_workspace(int nD)
{
    return nD < 1 ? 0 : lrs_workspace(nD);
}

rbsog_status rbsog_longrange_force(const double *r, const double *q, int n_atoms, const double box[3], const int *m,
                                   const int *cr, const int *cnr, int nD, const double *rho, int P, double Sr,
                                   double Snr, double ke, double *F, double *est, void *work, int precision,
                                   void *stream)
{
    if (!box || !m || !cr || !rho || !work || n_atoms < 0 || nD < 1 || P < 1 || (n_atoms > 0 && (!r || !q || !F)) ||
        (precision != 0 && precision != 1) || !(Sr > 0) || (cnr && !(Snr > 0)))
        return fail(nullptr, RBSOG_EINVAL, "rbsog_longrange_force: bad argument");
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 0)) return fail(nullptr, RBSOG_EBOX, "rbsog_longrange_force: box edge <= 0");
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = lr_force_stateless(r, q, n_atoms, box, m, cr, cnr, nD, rho, P, Sr, Snr, ke, F, est, work,
                                       precision, cs);
    if (e == cudaSuccess && est) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess)
        return fail(nullptr, RBSOG_ECUDA, std::string("rbsog_longrange_force: ") + cudaGetErrorString(e));
    return RBSOG_OK;
}

}  // extern "C"
