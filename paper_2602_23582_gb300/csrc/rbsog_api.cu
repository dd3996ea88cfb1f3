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
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/rbsog.h"
#include "internal.h"

using namespace rbsog;

namespace {

constexpr double kKB = 0.0019872067;                         // kcal/(mol K)
constexpr double kFtm2v = 1.0 / 48.88821291 / 48.88821291;   // (kcal/mol/A)/(g/mol) -> A/fs^2
constexpr double kNktv2p = 68568.415;                        // atm per kcal/(mol A^3)

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
};

}  // namespace

struct rbsog_ctx {
    rbsog_params prm{};
    int S = 0, N = 0, C = 0, Dcap = 0, nchunks = 0, nmol = 0, nmchunks = 0, item_cap = 0;
    cudaStream_t st = nullptr, st2 = nullptr;
    bool own_st = false, own_st2 = false;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::string err;
    std::vector<int> h_atom0, h_n, h_cell0, h_ncap_total, h_coupling;
    std::vector<void *> allocs;
    // device
    DevSys *sys = nullptr;
    double *r = nullptr, *p = nullptr, *F = nullptr, *q = nullptr, *mass = nullptr;
    int *type = nullptr, *mol = nullptr, *atom_sys = nullptr, *cell = nullptr, *rank = nullptr;
    float4 *locf = nullptr, *pos4 = nullptr;
    double4 *locd = nullptr, *posd = nullptr;
    uint4 *su = nullptr;
    int *count = nullptr, *start = nullptr, *sidx = nullptr, *cell_sys = nullptr;
    float2 *qt = nullptr;
    int2 *aux = nullptr, *items = nullptr;
    int *chunk_sys = nullptr, *chunk_a0 = nullptr, *chunk_n = nullptr, *first_chunk = nullptr, *nchunk_sys = nullptr;
    int *mchunk_sys = nullptr, *mchunk_m0 = nullptr, *mchunk_n = nullptr, *mchunk_first = nullptr, *mchunk_count = nullptr;
    int *b_start = nullptr, *a_start = nullptr, *e_start = nullptr, *bonds = nullptr, *angles = nullptr, *excl = nullptr;
    double *bk = nullptr, *br0 = nullptr, *ak = nullptr, *at0 = nullptr;
    double *pair_part = nullptr, *lr_out = nullptr, *mol_part = nullptr, *kin_part = nullptr, *sysred = nullptr;
    double *self_e = nullptr;
    double4 *fpart = nullptr;   // pair forces per dz plane (FP32 build reads it as float4)
    double *pair_red = nullptr; // pair records reduced to kPairRedBlocks per system
    double *inv_m = nullptr, *sdv = nullptr;   // per-atom integrator constants
    double2 *ljd = nullptr;     // LJ blocks per system
    float2 *ljf = nullptr, *ljf_lo = nullptr;
    int *mr = nullptr, *mnr = nullptr, *D = nullptr, *cr = nullptr, *cnr = nullptr;
    int4 *pm = nullptr;
    double *pw = nullptr, *pg = nullptr, *pu = nullptr, *pun = nullptr;
    double *sk_part = nullptr, *rho = nullptr;
    ModeCoef *coef = nullptr;
    unsigned long long *d_step = nullptr;
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
    std::vector<std::string> t_names;
    std::vector<cudaEvent_t> t_events;
    std::vector<double> t_ms;
};

namespace {

thread_local std::string g_create_err;   // error text of a failed rbsog_create

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

template <typename T>
bool dalloc(rbsog_ctx *c, T *&ptr, size_t n)
{
    if (n == 0) n = 1;
    void *v = nullptr;
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
void enqueue_eval(rbsog_ctx *c, int kick, int box_kick, int energy)
{
    const int prec = c->prm.precision;
    record(c, "start");
    launch_box_prep(c->b, c->st);
    record(c, "box_prep");
    cudaEventRecord(c->ev_fork, c->st);
    cudaStreamWaitEvent(c->st2, c->ev_fork, 0);
    launch_sampler(c->b, c->sa, c->mr, c->mnr, c->D, c->cr, c->cnr, c->pm, c->pw, c->pg, c->pu, c->pun,
                   c->Dcap, c->st2);
    cudaEventRecord(c->ev_join, c->st2);
    launch_bin(c->b, c->a, prec, c->st);
    record(c, "bin");
    launch_scan(c->b, c->a, c->st);
    record(c, "scan");
    launch_scatter_sort(c->b, c->a, prec, c->st);
    record(c, "scatter_sort");
    // in a graph capture: event-record nodes around the pair kernel (external
    // records, not dependencies), retargeted per launch by arm_pair_trace
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->st, &cap);
    const bool trace = cap == cudaStreamCaptureStatusActive && c->ev_pair_ph[0] && c->ev_pair_ph[1];
    if (trace) cudaEventRecordWithFlags(c->ev_pair_ph[0], c->st, cudaEventRecordExternal);
    launch_pair(c->b, c->a, prec, c->pcf, c->pcd, energy, c->pair_part, c->st);
    if (trace) cudaEventRecordWithFlags(c->ev_pair_ph[1], c->st, cudaEventRecordExternal);
    record(c, "pair");
    cudaStreamWaitEvent(c->st, c->ev_join, 0);
    record(c, "sampler_join");
    launch_sk(c->b, c->a, prec, c->D, c->Dcap, c->sk_part, c->st);
    record(c, "structure_factor");
    launch_estimate(c->b, c->first_chunk, c->nchunk_sys, c->D, c->cr, c->cnr, c->Dcap, c->prm.P, c->prm.ke,
                    c->sk_part, c->rho, c->coef, c->lr_out, c->st);
    record(c, "estimate");
    launch_lr_force(c->b, c->a, prec, c->coef, c->Dcap, c->st);
    record(c, "lr_force");
    launch_mol(c->b, c->a, c->m, c->sc, c->mol_part, prec, c->st);
    record(c, "molecules");
    launch_kick_kinetic(c->b, c->a, c->ia, kick, c->kin_part, c->st);
    record(c, "kick_kinetic");
    launch_reduce_pair(c->b, c->pair_part, c->pair_red, c->st);
    launch_finalize(c->b, c->pair_red, c->lr_out, c->mol_part, c->mchunk_first, c->mchunk_count, c->kin_part,
                    c->first_chunk, c->nchunk_sys, c->self_e, c->ia, box_kick, c->sysred, c->d_step, c->st);
    record(c, "finalize");
}

void enqueue_npt_step(rbsog_ctx *c, int energy)
{
    launch_box_half(c->b, c->ia, c->sysred, c->st);
    launch_atom_update(c->b, c->a, c->ia, c->st);
    enqueue_eval(c, 1, 1, energy);
}

rbsog_status check_flags(rbsog_ctx *c)
{
    std::vector<DevSys> h(c->S);
    cudaError_t e = cudaMemcpyAsync(h.data(), c->sys, sizeof(DevSys) * c->S, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "device");
    for (int s = 0; s < c->S; ++s) {
        if (h[s].flags & FLAG_BOX)
            return fail(c, RBSOG_EBOX, "system " + std::to_string(s) + ": box edge below " +
                                           std::to_string(2 * c->prm.cell_sub + 1) + " cells of r_c/sub");
        if (h[s].flags & FLAG_OVERFLOW)
            return fail(c, RBSOG_EOVERFLOW, "system " + std::to_string(s) + ": a cell holds more than " +
                                                std::to_string(kCellCap) + " atoms");
        if (h[s].flags & FLAG_NONFINITE)
            return fail(c, RBSOG_ENONFINITE, "system " + std::to_string(s) + ": non-finite energy or virial");
    }
    return RBSOG_OK;
}

rbsog_status fill_results(rbsog_ctx *c, rbsog_result *res)
{
    std::vector<double> h((size_t)c->S * kRed);
    cudaError_t e = cudaMemcpyAsync(h.data(), c->sysred, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    unsigned long long step = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&step, c->d_step, sizeof(step), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "results");
    static const int sym[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};   // 3x3 row-major from xx yy zz xy xz yz
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
        r.n_distinct_modes = (int)o[55];
        r.n_accept_r = (int)o[56];
        r.n_accept_nr = (int)o[57];
        r.step = step;
    }
    return RBSOG_OK;
}

void free_ctx(rbsog_ctx *c)
{
    if (!c) return;
    for (auto g : c->graph)
        if (g) cudaGraphExecDestroy(g);
    for (auto g : c->graph_src)
        if (g) cudaGraphDestroy(g);
    for (auto e : c->ring_s) cudaEventDestroy(e);
    for (auto e : c->ring_e) cudaEventDestroy(e);
    for (auto e : c->ev_pair_ph)
        if (e) cudaEventDestroy(e);
    for (auto e : c->t_events) cudaEventDestroy(e);
    for (void *v : c->allocs) cudaFree(v);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->own_st2 && c->st2) cudaStreamDestroy(c->st2);
    if (c->own_st && c->st) cudaStreamDestroy(c->st);
    delete c;
}

rbsog_status validate(const rbsog_params *p, int S, const rbsog_system_desc *sy)
{
    if (!p || S <= 0 || !sy) return RBSOG_EINVAL;
    if (!(p->rc > 0) || !(p->b > 1) || !(p->sigma > 0) || p->M < 1 || p->M > kMaxGauss ||
        p->M_energy < p->M || p->M_energy > kMaxGauss || p->P < 1 || p->P > kMaxP ||
        p->sampler < 0 || p->sampler > 2 || (p->precision != 0 && p->precision != 1) ||
        (p->cell_sub < 0 || p->cell_sub > 2) || p->coupling < 0 || p->coupling > 2 || p->thermo_every < 0)
        return RBSOG_EINVAL;
    for (int s = 0; s < S; ++s) {
        const rbsog_system_desc &d = sy[s];
        if (d.n_atoms < 1 || !d.q || !d.mass || !d.type || !d.mol || !d.r0 || d.ntypes < 1 ||
            d.ntypes > kMaxTypes || !d.lj_eps || !d.lj_sig)
            return RBSOG_EINVAL;
        for (int a = 0; a < 3; ++a)
            if (!(d.box[a] > 0)) return RBSOG_EBOX;
        for (int i = 0; i < d.n_atoms; ++i)
            if (!(d.mass[i] > 0) || !std::isfinite(d.mass[i])) return RBSOG_EINVAL;
    }
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

int rbsog_n_atoms(const rbsog_ctx *ctx) { return ctx ? ctx->N : 0; }

rbsog_status rbsog_system_range(const rbsog_ctx *ctx, int s, int *atom0, int *n)
{
    if (!ctx || s < 0 || s >= ctx->S) return RBSOG_EINVAL;
    if (atom0) *atom0 = ctx->h_atom0[s];
    if (n) *n = ctx->h_n[s];
    return RBSOG_OK;
}

void rbsog_destroy(rbsog_ctx *ctx) { free_ctx(ctx); }

rbsog_status rbsog_create(const rbsog_params *params, int n_systems, const rbsog_system_desc *systems,
                          void *stream, rbsog_ctx **out)
{
    if (!out) return RBSOG_EINVAL;
    *out = nullptr;
    rbsog_status vs = validate(params, n_systems, systems);
    if (vs != RBSOG_OK) return vs;
    rbsog_ctx *c = new (std::nothrow) rbsog_ctx();
    if (!c) return RBSOG_ENOMEM;
    try {
        c->prm = *params;
        if (c->prm.cell_sub == 0) {
            // cells of r_c/2 when a box edge leaves little room above 3 r_c (the
            // box fluctuates in NPT), else cells of r_c
            c->prm.cell_sub = 1;
            for (int k = 0; k < n_systems; ++k)
                for (int a2 = 0; a2 < 3; ++a2)
                    if (systems[k].box[a2] < 3.3 * c->prm.rc) c->prm.cell_sub = 2;
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
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
        cudaEventCreate(&c->ev_pair_ph[0]);
        cudaEventCreate(&c->ev_pair_ph[1]);
        c->Dcap = (P.sampler == RBSOG_SAMPLER_IID) ? 2 * P.P : P.P + 1;

        // ---- host layout
        const int S = c->S;
        std::vector<DevSys> hsys(S);
        std::vector<int> atom_sys, cell_sys, chunk_sys, chunk_a0, chunk_n, first_chunk(S), nchunk(S);
        std::vector<int> mchunk_sys, mchunk_m0, mchunk_n, mchunk_first(S), mchunk_count(S);
        std::vector<double> r, p, q, mass, self_e(2 * S);
        std::vector<int> type, mol;
        std::vector<int> b_start{0}, a_start{0}, e_start{0}, bonds, angles, excl;
        std::vector<double> bk, br0, ak, at0;
        std::vector<double2> ljd;
        std::vector<double> inv_m, sdv;
        const double c_atom = std::exp(-P.gamma * P.dt);
        std::vector<float2> ljf, ljf_lo;
        int N = 0, C = 0, nmol = 0, item_cap = 0;
        std::vector<double> w, s, wt, st;
        const int MM = std::max(P.M, P.M_energy);
        sog_terms(P, MM, w, s, wt, st);
        c->h_atom0.resize(S); c->h_n.resize(S); c->h_cell0.resize(S); c->h_ncap_total.resize(S);
        for (int k = 0; k < S; ++k) {
            const rbsog_system_desc &d = systems[k];
            DevSys &ds = hsys[k];
            std::memset(&ds, 0, sizeof(ds));
            int ncap_t = 1;
            for (int a = 0; a < 3; ++a) {
                ds.L[a] = d.box[a];
                int n = (int)std::floor(d.box[a] * P.cell_sub / P.rc);
                if (n < 2 * P.cell_sub + 1) {
                    rbsog_status rr = fail(c, RBSOG_EBOX, "system " + std::to_string(k) + ": box edge " +
                                                              std::to_string(d.box[a]) + " too small for the cell stencil");
                    free_ctx(c);
                    return rr;
                }
                int cap = (int)std::floor(d.box[a] * 1.15 * P.cell_sub / P.rc);
                ds.ncap[a] = std::max(cap, n);
                ncap_t *= ds.ncap[a];
            }
            ds.V = d.box[0] * d.box[1] * d.box[2];
            ds.cell0 = C;
            ds.ncell_cap_total = ncap_t;
            // pair work items: at most one partial 32-atom group per cell; a
            // multiple of kPairWarps so that no pair-kernel block spans two systems
            ds.item0 = item_cap;
            ds.item_cap = ((d.n_atoms + 31) / 32 + ncap_t + kPairWarps - 1) / kPairWarps * kPairWarps;
            item_cap += ds.item_cap;
            ds.atom0 = N;
            ds.n = d.n_atoms;
            ds.coupling = P.coupling == RBSOG_COUPLE_SEMI_ISO ? 1 : 0;
            ds.rng_id = d.rng_id;
            // LJ block of this system: (4 eps sig^12, 4 eps sig^6) per type pair
            ds.ntypes = d.ntypes;
            ds.lj0 = (int)ljd.size();
            for (int t = 0; t < d.ntypes * d.ntypes; ++t) {
                const double eps = d.lj_eps[t], sg = d.lj_sig[t];
                const double s6 = sg * sg * sg * sg * sg * sg;
                ljd.push_back(make_double2(4.0 * eps * s6 * s6, 4.0 * eps * s6));
                ljf.push_back(make_float2((float)ljd.back().x, (float)ljd.back().y));
                ljf_lo.push_back(make_float2((float)(ljd.back().x - (double)ljf.back().x),
                                             (float)(ljd.back().y - (double)ljf.back().y)));
            }
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
            c->h_atom0[k] = N; c->h_n[k] = d.n_atoms; c->h_cell0[k] = C; c->h_ncap_total[k] = ncap_t;
            for (int i = 0; i < ncap_t; ++i) cell_sys.push_back(k);
            C += ncap_t;
            // atoms
            double sq = 0.0;
            for (int i = 0; i < d.n_atoms; ++i) {
                atom_sys.push_back(k);
                for (int a = 0; a < 3; ++a) {
                    r.push_back(d.r0[3 * i + a]);
                    p.push_back(d.v0 ? d.v0[3 * i + a] * d.mass[i] : 0.0);
                }
                q.push_back(d.q[i]);
                mass.push_back(d.mass[i]);
                inv_m.push_back(1.0 / d.mass[i]);
                sdv.push_back(std::sqrt((1.0 - c_atom * c_atom) * d.mass[i] * kKB * P.T * kFtm2v));
                if (d.type[i] < 0 || d.type[i] >= d.ntypes) {
                    rbsog_status rr = fail(c, RBSOG_EINVAL, "atom type out of range");
                    free_ctx(c);
                    return rr;
                }
                type.push_back(d.type[i]);
                mol.push_back(d.mol[i]);
                sq += d.q[i] * d.q[i];
            }
            // App. A: U_self = ln b / (sqrt(2 pi) sigma) (omega + (1 - b^{-(M-1)})/(b - 1)) sum q^2
            self_e[2 * k] = P.ke * std::log(P.b) / (std::sqrt(2.0 * kPi) * P.sigma) *
                            (P.omega + (1.0 - std::pow(P.b, -(P.M_energy - 1.0))) / (P.b - 1.0)) * sq;
            // FP32 build: the constant part sum_excl ke q_i q_j F_E(0) of the exclusion energy
            if (P.precision == RBSOG_FP32) {
                double fe0 = 0.0, sx = 0.0;
                for (int l = 0; l < P.M_energy; ++l) fe0 += w[l];
                for (int e2 = 0; e2 < d.n_excl; ++e2) sx += d.q[d.excl[2 * e2]] * d.q[d.excl[2 * e2 + 1]];
                self_e[2 * k + 1] = P.ke * fe0 * sx;
            }
            // chunks
            first_chunk[k] = (int)chunk_sys.size();
            for (int a0 = 0; a0 < d.n_atoms; a0 += kChunk) {
                chunk_sys.push_back(k);
                chunk_a0.push_back(N + a0);
                chunk_n.push_back(std::min(kChunk, d.n_atoms - a0));
            }
            nchunk[k] = (int)chunk_sys.size() - first_chunk[k];
            // molecules: maximal runs of equal mol id
            std::vector<int> mol_of(d.n_atoms);
            std::vector<int> mstart;
            for (int i = 0; i < d.n_atoms; ++i) {
                if (i == 0 || d.mol[i] != d.mol[i - 1]) mstart.push_back(i);
                mol_of[i] = (int)mstart.size() - 1;
            }
            const int nm = (int)mstart.size();
            std::vector<std::vector<int>> mb(nm), ma(nm), me(nm);
            auto same = [&](int i, int j) { return i >= 0 && j >= 0 && i < d.n_atoms && j < d.n_atoms && mol_of[i] == mol_of[j]; };
            for (int e2 = 0; e2 < d.n_bonds; ++e2) {
                int i = d.bonds[2 * e2], j = d.bonds[2 * e2 + 1];
                if (!same(i, j)) { rbsog_status rr = fail(c, RBSOG_EINVAL, "a bond spans two molecules"); free_ctx(c); return rr; }
                mb[mol_of[i]].push_back(e2);
            }
            for (int e2 = 0; e2 < d.n_angles; ++e2) {
                int i = d.angles[3 * e2], j = d.angles[3 * e2 + 1], kk = d.angles[3 * e2 + 2];
                if (!same(i, j) || !same(j, kk)) { rbsog_status rr = fail(c, RBSOG_EINVAL, "an angle spans two molecules"); free_ctx(c); return rr; }
                ma[mol_of[i]].push_back(e2);
            }
            for (int e2 = 0; e2 < d.n_excl; ++e2) {
                int i = d.excl[2 * e2], j = d.excl[2 * e2 + 1];
                if (!same(i, j)) { rbsog_status rr = fail(c, RBSOG_EINVAL, "an exclusion spans two molecules"); free_ctx(c); return rr; }
                me[mol_of[i]].push_back(e2);
            }
            mchunk_first[k] = (int)mchunk_sys.size();
            for (int m0 = 0; m0 < nm; m0 += kMolChunk) {
                mchunk_sys.push_back(k);
                mchunk_m0.push_back(nmol + m0);
                mchunk_n.push_back(std::min(kMolChunk, nm - m0));
            }
            mchunk_count[k] = (int)mchunk_sys.size() - mchunk_first[k];
            for (int mm = 0; mm < nm; ++mm) {
                for (int e2 : mb[mm]) {
                    bonds.push_back(N + d.bonds[2 * e2]); bonds.push_back(N + d.bonds[2 * e2 + 1]);
                    bk.push_back(d.bond_k[e2]); br0.push_back(d.bond_r0[e2]);
                }
                for (int e2 : ma[mm]) {
                    for (int t = 0; t < 3; ++t) angles.push_back(N + d.angles[3 * e2 + t]);
                    ak.push_back(d.angle_k[e2]); at0.push_back(d.angle_t0[e2]);
                }
                for (int e2 : me[mm]) {
                    excl.push_back(N + d.excl[2 * e2]); excl.push_back(N + d.excl[2 * e2 + 1]);
                }
                b_start.push_back((int)bk.size());
                a_start.push_back((int)ak.size());
                e_start.push_back((int)excl.size() / 2);
            }
            nmol += nm;
            N += d.n_atoms;
        }
        if (N >= (1 << 25)) {
            // the pair kernel's queue packs a neighbour index into 25 bits
            rbsog_status rr = fail(c, RBSOG_EUNSUPPORTED, "more than 2^25 - 1 atoms in one context");
            free_ctx(c);
            return rr;
        }
        c->N = N; c->C = C; c->nmol = nmol; c->item_cap = item_cap;
        c->nchunks = (int)chunk_sys.size();
        c->nmchunks = (int)mchunk_sys.size();

        // ---- device buffers
        bool ok = upload(c, c->sys, hsys) && upload(c, c->r, r) && upload(c, c->p, p) && upload(c, c->q, q) &&
                  upload(c, c->mass, mass) && upload(c, c->type, type) && upload(c, c->mol, mol) &&
                  upload(c, c->atom_sys, atom_sys) && upload(c, c->cell_sys, cell_sys) &&
                  upload(c, c->chunk_sys, chunk_sys) && upload(c, c->chunk_a0, chunk_a0) &&
                  upload(c, c->chunk_n, chunk_n) && upload(c, c->first_chunk, first_chunk) &&
                  upload(c, c->nchunk_sys, nchunk) && upload(c, c->mchunk_sys, mchunk_sys) &&
                  upload(c, c->mchunk_m0, mchunk_m0) && upload(c, c->mchunk_n, mchunk_n) &&
                  upload(c, c->mchunk_first, mchunk_first) && upload(c, c->mchunk_count, mchunk_count) &&
                  upload(c, c->b_start, b_start) && upload(c, c->a_start, a_start) && upload(c, c->e_start, e_start) &&
                  upload(c, c->bonds, bonds) && upload(c, c->angles, angles) && upload(c, c->excl, excl) &&
                  upload(c, c->bk, bk) && upload(c, c->br0, br0) && upload(c, c->ak, ak) && upload(c, c->at0, at0) &&
                  upload(c, c->self_e, self_e) && dalloc(c, c->F, 3 * (size_t)N) && dalloc(c, c->cell, N) &&
                  dalloc(c, c->rank, N) && dalloc(c, c->sidx, N) && dalloc(c, c->count, C) &&
                  dalloc(c, c->start, C + 1) && dalloc(c, c->items, item_cap) &&
                  dalloc(c, c->pair_part, (size_t)item_cap * (2 * P.cell_sub + 1) / kPairWarps * kPairRec) &&
                  dalloc(c, c->fpart, (size_t)N * (2 * P.cell_sub + 1)) &&
                  dalloc(c, c->pair_red, (size_t)S * kPairRedBlocks * kPairRec) &&
                  dalloc(c, c->lr_out, (size_t)S * 16) && dalloc(c, c->mol_part, (size_t)c->nmchunks * 15) &&
                  dalloc(c, c->kin_part, (size_t)c->nchunks * kKinSplit * 6) && dalloc(c, c->sysred, (size_t)S * kRed) &&
                  dalloc(c, c->mr, (size_t)S * P.P * 3) && dalloc(c, c->mnr, (size_t)S * P.P * 3) &&
                  dalloc(c, c->D, (size_t)S * c->Dcap * 3) && dalloc(c, c->cr, (size_t)S * c->Dcap) &&
                  dalloc(c, c->cnr, (size_t)S * c->Dcap) && dalloc(c, c->pm, (size_t)S * P.P) &&
                  dalloc(c, c->pw, (size_t)S * P.P) && dalloc(c, c->pg, (size_t)S * P.P) &&
                  dalloc(c, c->pu, (size_t)S * P.P) && dalloc(c, c->pun, (size_t)S * P.P) &&
                  dalloc(c, c->sk_part, (size_t)c->nchunks * c->Dcap * 2) &&
                  dalloc(c, c->rho, (size_t)S * c->Dcap * 2) && dalloc(c, c->coef, (size_t)S * c->Dcap) &&
                  dalloc(c, c->d_step, 1) && upload(c, c->ljd, ljd) && upload(c, c->ljf, ljf) && upload(c, c->ljf_lo, ljf_lo) &&
                  upload(c, c->inv_m, inv_m) && upload(c, c->sdv, sdv);
        if (ok) {
            if (P.precision == 1)
                ok = dalloc(c, c->locf, N) && dalloc(c, c->pos4, N) && dalloc(c, c->qt, N) && dalloc(c, c->su, N);
            else
                ok = dalloc(c, c->locd, N) && dalloc(c, c->posd, N) && dalloc(c, c->aux, N);
        }
        if (!ok) {
            free_ctx(c);
            return RBSOG_ENOMEM;
        }

        // ---- constants
        c->sc.M = P.M; c->sc.ME = P.M_energy; c->sc.rc = P.rc; c->sc.ke = P.ke;
        for (int l = 0; l < MM; ++l) { c->sc.w[l] = w[l]; c->sc.s[l] = s[l]; c->sc.wt[l] = wt[l]; c->sc.st[l] = st[l]; }
        c->pcf.M = c->pcd.M = P.M;
        c->pcf.ME = c->pcd.ME = P.M_energy;
        c->pcf.rc2 = (float)(P.rc * P.rc); c->pcd.rc2 = P.rc * P.rc; c->pcf.rc2d = P.rc * P.rc;
        c->pcf.rc2_hi = (float)(P.rc * P.rc * (1.0 + 1e-5));
        c->pcf.rc2_lo = (float)(P.rc * P.rc * (1.0 - 1e-5));
        c->pcf.ke = (float)P.ke; c->pcd.ke = P.ke;
        for (int l = 0; l < MM; ++l) {
            c->pcd.inv_s2[l] = 1.0 / (s[l] * s[l]);
            c->pcd.w[l] = w[l];
            c->pcd.wt[l] = l < P.M ? wt[l] : 0.0;
        }
        {
            // FP32 split: Gaussians with s_l >= 2.5 r_c go into a Taylor tail in u = r^2
            const double swide = 2.5 * P.rc, log2e = 1.4426950408889634;
            int nff = 0, nfe = 0;
            while (nff < P.M && st[nff] < swide) ++nff;
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
            // sum_l w_l e^{-u/s_l^2} = sum_k u^k sum_l w_l (-1/s_l^2)^k / k!
            double te0 = 0.0;
            for (int k = 0; k <= kTail; ++k) {
                double tk = 0.0, ek = 0.0, fact = 1.0;
                for (int i = 2; i <= k; ++i) fact *= i;
                for (int l = nff; l < P.M; ++l) tk += wt[l] * std::pow(-1.0 / (st[l] * st[l]), k) / fact;
                for (int l = nfe; l < P.M_energy; ++l) ek += w[l] * std::pow(-1.0 / (s[l] * s[l]), k) / fact;
                c->pcf.tt[k] = (float)tk;
                c->pcf.te[k] = k == 0 ? 0.f : (float)ek;
                if (k == 0) te0 = ek;
            }
            c->pcf.te0 = te0;
        }
        // LJ: one ntypes x ntypes block per system (uploaded with the buffers above)
        // sampler (the same expressions as the paper's formulas, FP64 on the host)
        c->sa.P = P.P; c->sa.M = P.M; c->sa.kind = P.sampler; c->sa.seed = P.seed; c->sa.step = c->d_step;
        const double pi15 = std::pow(kPi, 1.5);
        for (int l = 0; l < P.M; ++l) {
            double s5 = st[l] * st[l] * st[l] * st[l] * st[l];
            c->sa.wt[l] = wt[l]; c->sa.st[l] = st[l];
            c->sa.cr[l] = pi15 * wt[l] * s5;
            c->sa.cn[l] = pi15 * wt[l] * s5 * st[l] * st[l];
            c->sa.st2q[l] = st[l] * st[l] * 0.25;
        }
        c->sa.sig_u = 1.0 / (std::sqrt(2.0) * kPi * st[0]);
        c->ia.dt = P.dt; c->ia.T = P.T; c->ia.Pext = P.P_ext; c->ia.gamma = P.gamma; c->ia.gamma_box = P.gamma_box;
        c->ia.kB = kKB; c->ia.ftm2v = kFtm2v; c->ia.nktv2p = kNktv2p; c->ia.seed = P.seed; c->ia.step = c->d_step;
        c->ia.c_atom = std::exp(-P.gamma * P.dt);
        c->ia.inv_m = c->inv_m; c->ia.sdv = c->sdv;
        c->ia.noise_f32 = P.precision == RBSOG_FP32 ? 1 : 0;

        c->b.S = S; c->b.N = N; c->b.C = C; c->b.sub = P.cell_sub; c->b.rc = P.rc; c->b.sys = c->sys;
        c->b.atom_sys = c->atom_sys; c->b.cell_sys = c->cell_sys; c->b.chunk_sys = c->chunk_sys;
        c->b.chunk_a0 = c->chunk_a0; c->b.chunk_n = c->chunk_n; c->b.nchunks = c->nchunks;
        c->b.item_cap = item_cap;
        c->a.r = c->r; c->a.p = c->p; c->a.F = c->F; c->a.q = c->q; c->a.mass = c->mass; c->a.type = c->type;
        c->a.mol = c->mol; c->a.cell = c->cell; c->a.rank = c->rank; c->a.locf = c->locf; c->a.locd = c->locd;
        c->a.su = c->su; c->a.count = c->count; c->a.start = c->start; c->a.sidx = c->sidx; c->a.pos4 = c->pos4;
        c->a.qt = c->qt; c->a.posd = c->posd; c->a.aux = c->aux; c->a.items = c->items;
        c->a.fpartd = c->fpart; c->a.fpart4 = reinterpret_cast<float4 *>(c->fpart);
        c->a.ljd = c->ljd; c->a.ljf = c->ljf; c->a.ljf_lo = c->ljf_lo;
        c->m.nmol = nmol; c->m.b_start = c->b_start; c->m.a_start = c->a_start; c->m.e_start = c->e_start;
        c->m.bonds = c->bonds; c->m.bk = c->bk; c->m.br0 = c->br0; c->m.angles = c->angles; c->m.ak = c->ak;
        c->m.at0 = c->at0; c->m.excl = c->excl; c->m.mchunk_sys = c->mchunk_sys; c->m.mchunk_m0 = c->mchunk_m0;
        c->m.mchunk_n = c->mchunk_n; c->m.nmchunks = c->nmchunks;

        e = prepare_sampler(P.P);
        if (e == cudaSuccess) e = prepare_pair();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { rbsog_status rr = cuda_fail(c, e, "create"); free_ctx(c); return rr; }
        // the first evaluation (counter 0) primes forces, virial and kinetic tensor
        unsigned long long minus1 = ~0ull;
        cudaMemcpyAsync(c->d_step, &minus1, sizeof(minus1), cudaMemcpyHostToDevice, c->st);
        launch_clear_flags(c->b, c->st);
        enqueue_eval(c, 0, 0, 1);
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

rbsog_status rbsog_set_box(rbsog_ctx *c, int s, const double box[3], int rescale)
{
    if (!c || s < 0 || s >= c->S || !box) return RBSOG_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 0) || (int)std::floor(box[a] * c->prm.cell_sub / c->prm.rc) < 2 * c->prm.cell_sub + 1)
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

rbsog_status rbsog_step(rbsog_ctx *c, uint64_t step, double *forces, int on_device, rbsog_result *res)
{
    if (!c) return RBSOG_EINVAL;
    unsigned long long prev = (unsigned long long)step - 1ull;
    cudaError_t e = cudaMemcpyAsync(c->d_step, &prev, sizeof(prev), cudaMemcpyHostToDevice, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "step");
    for (auto ev : c->t_events) cudaEventDestroy(ev);
    c->t_events.clear();
    c->t_names.clear();
    launch_clear_flags(c->b, c->st);
    enqueue_eval(c, 0, 0, 1);
    c->h_step = (unsigned long long)step;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
    if (forces) {
        e = cudaMemcpyAsync(forces, c->F, 3 * sizeof(double) * c->N,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st);
        if (e != cudaSuccess) return cuda_fail(c, e, "forces");
    }
    rbsog_status fs = check_flags(c);
    if (fs != RBSOG_OK) return fs;
    if (c->timing) {
        c->t_ms.clear();
        for (size_t k = 1; k < c->t_events.size(); ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, c->t_events[k - 1], c->t_events[k]);
            c->t_ms.push_back(ms);
        }
    }
    if (res) return fill_results(c, res);
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

void *rbsog_stream(rbsog_ctx *c) { return c ? (void *)c->st : nullptr; }

rbsog_status rbsog_run(rbsog_ctx *c, int nsteps, rbsog_result *last)
{
    if (!c || nsteps < 0) return RBSOG_EINVAL;
    launch_clear_flags(c->b, c->st);
    rbsog_status rs = run_steps(c, nsteps, true);
    if (rs != RBSOG_OK) return rs;
    rbsog_status fs = check_flags(c);
    if (fs != RBSOG_OK) return fs;
    if (last) return fill_results(c, last);
    return RBSOG_OK;
}

rbsog_status rbsog_get_state(rbsog_ctx *c, void *buf, size_t *len)
{
    if (!c || !len) return RBSOG_EINVAL;
    const size_t need = sizeof(uint64_t) * 2 + 6 * sizeof(double) * (size_t)c->N + sizeof(DevSys) * c->S +
                        3 * sizeof(double) * (size_t)c->N + sizeof(double) * (size_t)c->S * kRed;
    if (!buf) { *len = need; return RBSOG_OK; }
    if (*len < need) return RBSOG_EINVAL;
    unsigned long long step = 0;
    cudaError_t e = cudaMemcpyAsync(&step, c->d_step, sizeof(step), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    uint64_t hdr[2] = {(uint64_t)step, (uint64_t)c->N};
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
    if (e == cudaSuccess) e = cudaMemcpy(c->d_step, &step, sizeof(step), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_state");
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

}  // extern "C"
