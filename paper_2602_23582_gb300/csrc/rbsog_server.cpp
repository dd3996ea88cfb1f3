// rbsog_server.cpp -- request loop of the served path, built on the pool API
// of rbsog.h (host code only).
//
// Requests (a system and a number of NPT steps) wait in a FIFO queue.  Each
// call of rbsog_server_pump is one round:
//   1. finished slots are unloaded and their results stored under the ticket;
//   2. queued requests are admitted in arrival order into free slots whose
//      capacities fit them (first fit; a request that fits no slot of the
//      pool is refused at submission), and the new slots are primed with a
//      force evaluation;
//   3. every running slot advances up to `max_steps` NPT steps in the same
//      kernel launches (one CUDA graph per step), each step timed with CUDA
//      events on the context stream.
// The pool is sized at creation so that its device memory fits a fraction of
// the free HBM; admission is then a matter of free slots.  All per-system
// state (positions, momenta, box, box momentum, Philox counter) stays on the
// device from admission to retirement.
#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/rbsog.h"

namespace {

// Owned host copy of a system description.
struct SystemCopy {
    rbsog_system_desc d{};
    std::vector<double> q, mass, bond_k, bond_r0, angle_k, angle_t0, lj_eps, lj_sig, r0, v0;
    std::vector<int> type, mol, bonds, angles, excl;

    explicit SystemCopy(const rbsog_system_desc &s)
    {
        const int n = s.n_atoms;
        q.assign(s.q, s.q + n);
        mass.assign(s.mass, s.mass + n);
        type.assign(s.type, s.type + n);
        mol.assign(s.mol, s.mol + n);
        r0.assign(s.r0, s.r0 + 3 * (size_t)n);
        if (s.v0) v0.assign(s.v0, s.v0 + 3 * (size_t)n);
        lj_eps.assign(s.lj_eps, s.lj_eps + s.ntypes * s.ntypes);
        lj_sig.assign(s.lj_sig, s.lj_sig + s.ntypes * s.ntypes);
        if (s.n_bonds > 0) {
            bonds.assign(s.bonds, s.bonds + 2 * (size_t)s.n_bonds);
            bond_k.assign(s.bond_k, s.bond_k + s.n_bonds);
            bond_r0.assign(s.bond_r0, s.bond_r0 + s.n_bonds);
        }
        if (s.n_angles > 0) {
            angles.assign(s.angles, s.angles + 3 * (size_t)s.n_angles);
            angle_k.assign(s.angle_k, s.angle_k + s.n_angles);
            angle_t0.assign(s.angle_t0, s.angle_t0 + s.n_angles);
        }
        if (s.n_excl > 0) excl.assign(s.excl, s.excl + 2 * (size_t)s.n_excl);
        d = s;
        d.q = q.data(); d.mass = mass.data(); d.type = type.data(); d.mol = mol.data();
        d.lj_eps = lj_eps.data(); d.lj_sig = lj_sig.data(); d.r0 = r0.data();
        d.v0 = v0.empty() ? nullptr : v0.data();
        d.bonds = bonds.empty() ? nullptr : bonds.data();
        d.bond_k = bond_k.empty() ? nullptr : bond_k.data();
        d.bond_r0 = bond_r0.empty() ? nullptr : bond_r0.data();
        d.angles = angles.empty() ? nullptr : angles.data();
        d.angle_k = angle_k.empty() ? nullptr : angle_k.data();
        d.angle_t0 = angle_t0.empty() ? nullptr : angle_t0.data();
        d.excl = excl.empty() ? nullptr : excl.data();
    }
};

struct Request {
    rbsog_status status = RBSOG_OK;   // RBSOG_OK, or why the system was stopped early
    long long ticket = 0;
    SystemCopy *sys = nullptr;
    int nsteps = 0;
    int slot = -1;
    bool done = false;
    std::vector<double> r, v;
    rbsog_result res{};
};

int molecules_of(const rbsog_system_desc &d)
{
    int nm = 0;
    for (int i = 0; i < d.n_atoms; ++i)
        if (i == 0 || d.mol[i] != d.mol[i - 1]) ++nm;
    return nm;
}

bool fits(const rbsog_slot_caps &c, const rbsog_system_desc &d)
{
    if (d.n_atoms > c.max_atoms || d.n_bonds > c.max_bonds || d.n_angles > c.max_angles ||
        d.n_excl > c.max_excl || d.ntypes > c.max_types || molecules_of(d) > c.max_molecules)
        return false;
    for (int a = 0; a < 3; ++a)
        if (d.box[a] > c.max_box[a]) return false;
    return true;
}

}  // namespace

struct rbsog_server {
    rbsog_ctx *ctx = nullptr;
    std::vector<rbsog_slot_caps> caps;     // per slot
    std::vector<long long> slot_ticket;    // -1: free
    std::deque<long long> queue;
    std::map<long long, Request> req;
    long long next_ticket = 1;
    std::vector<int> slot_atoms, slot_left;   // atoms and remaining steps of each slot's request
    // statistics
    std::vector<double> step_ms;
    double atom_steps = 0.0, gpu_ms = 0.0;
    int failed = 0;
    std::vector<cudaEvent_t> ev;
    std::string err;
};

extern "C" {

rbsog_status rbsog_server_create(const rbsog_params *params, int n_slots, const rbsog_slot_caps *caps,
                                 double hbm_fraction, void *stream, rbsog_server **out)
{
    if (!params || n_slots <= 0 || !caps || !out || !(hbm_fraction > 0) || hbm_fraction > 1) return RBSOG_EINVAL;
    *out = nullptr;
    rbsog_server *s = new (std::nothrow) rbsog_server();
    if (!s) return RBSOG_ENOMEM;
    // size the pool to the free HBM: the largest n <= n_slots whose pool fits
    // within hbm_fraction of the free memory at creation
    // (a failed query of the free memory is a CUDA error: no pool is sized on a guess)
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete s;
        return RBSOG_ECUDA;
    }
    const double budget = hbm_fraction * (double)free_b;
    int n = n_slots;
    rbsog_status st = RBSOG_ENOMEM;
    while (n >= 1) {
        size_t f0 = 0, f1 = 0, t = 0;
        if (cudaMemGetInfo(&f0, &t) != cudaSuccess) {
            st = RBSOG_ECUDA;
            break;
        }
        st = rbsog_pool_create(params, n, caps, stream, &s->ctx);
        if (st == RBSOG_OK) {
            if (cudaMemGetInfo(&f1, &t) != cudaSuccess) {
                rbsog_destroy(s->ctx);
                s->ctx = nullptr;
                st = RBSOG_ECUDA;
                break;
            }
            if ((double)(f0 - std::min(f0, f1)) <= budget) break;
            rbsog_destroy(s->ctx);
            s->ctx = nullptr;
            st = RBSOG_ENOMEM;
        } else if (st != RBSOG_ENOMEM) {
            break;
        }
        n = n * 3 / 4;                        // fewer slots, same classes in order
    }
    if (st != RBSOG_OK) {
        delete s;
        return st;
    }
    s->caps.assign(caps, caps + n);
    s->slot_ticket.assign(n, -1);
    s->slot_atoms.assign(n, 0);
    s->slot_left.assign(n, 0);
    *out = s;
    return RBSOG_OK;
}

void rbsog_server_destroy(rbsog_server *s)
{
    if (!s) return;
    for (auto e : s->ev) cudaEventDestroy(e);
    for (auto &kv : s->req) delete kv.second.sys;
    if (s->ctx) rbsog_destroy(s->ctx);
    delete s;
}

int rbsog_server_slots(const rbsog_server *s) { return s ? (int)s->caps.size() : 0; }

rbsog_ctx *rbsog_server_context(rbsog_server *s) { return s ? s->ctx : nullptr; }

rbsog_status rbsog_server_submit(rbsog_server *s, const rbsog_system_desc *sys, int nsteps, long long *ticket)
{
    if (!s || !sys || nsteps < 1 || !ticket) return RBSOG_EINVAL;
    bool any = false;
    for (const auto &c : s->caps) any = any || fits(c, *sys);
    if (!any) return RBSOG_EUNSUPPORTED;      // larger than every slot of the pool
    Request r;
    r.ticket = s->next_ticket++;
    r.sys = new (std::nothrow) SystemCopy(*sys);
    if (!r.sys) return RBSOG_ENOMEM;
    r.nsteps = nsteps;
    s->req[r.ticket] = std::move(r);
    s->queue.push_back(*ticket = s->next_ticket - 1);
    return RBSOG_OK;
}

rbsog_status rbsog_server_pump(rbsog_server *s, int max_steps, int *n_running, int *n_queued)
{
    if (!s || max_steps < 0) return RBSOG_EINVAL;
    const int S = (int)s->caps.size();
    std::vector<int> state(S), err(S);
    std::vector<unsigned long long> steps(S);
    rbsog_status st = rbsog_pool_state(s->ctx, state.data(), steps.data(), err.data());
    if (st != RBSOG_OK) return st;
    // 1. retire finished or failed slots
    for (int k = 0; k < S; ++k) {
        if (state[k] != 2 && state[k] != 3) continue;
        Request &r = s->req[s->slot_ticket[k]];
        r.status = (rbsog_status)err[k];
        if (state[k] == 3) {                  // count the steps it made, not the ones it was granted
            s->atom_steps -= (double)s->slot_atoms[k] * (r.nsteps - (long long)steps[k] - s->slot_left[k]);
            s->failed += 1;
        }
        r.r.resize(3 * (size_t)r.sys->d.n_atoms);
        r.v.resize(3 * (size_t)r.sys->d.n_atoms);
        st = rbsog_pool_unload(s->ctx, k, r.r.data(), r.v.data(), &r.res);
        if (st != RBSOG_OK) return st;
        r.done = true;
        r.slot = -1;
        delete r.sys;
        r.sys = nullptr;
        s->slot_ticket[k] = -1;
        s->slot_atoms[k] = 0;
        s->slot_left[k] = 0;
        state[k] = 0;
    }
    // 2. admit in arrival order, first fitting free slot
    bool admitted = false;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Request &r = s->req[*it];
        int slot = -1;
        for (int k = 0; k < S && slot < 0; ++k)
            if (s->slot_ticket[k] < 0 && fits(s->caps[k], r.sys->d)) slot = k;
        if (slot < 0) { ++it; continue; }
        st = rbsog_pool_load(s->ctx, slot, &r.sys->d, r.nsteps);
        if (st != RBSOG_OK) return st;
        r.slot = slot;
        s->slot_ticket[slot] = r.ticket;
        s->slot_atoms[slot] = r.sys->d.n_atoms;
        s->slot_left[slot] = r.nsteps;
        admitted = true;
        it = s->queue.erase(it);
    }
    if (admitted) {
        st = rbsog_pool_prime(s->ctx);
        if (st != RBSOG_OK) return st;
    }
    // 3. step the running slots together (a slot whose request completes
    // inside the round stops there, frozen on the device until retired)
    int running = 0;
    for (int k = 0; k < S; ++k)
        if (s->slot_ticket[k] >= 0 && s->slot_left[k] > 0) ++running;
    int most = 0;                             // no round longer than the longest remaining request
    for (int k = 0; k < S; ++k)
        if (s->slot_ticket[k] >= 0) most = std::max(most, s->slot_left[k]);
    max_steps = std::min(max_steps, most);
    if (running > 0 && max_steps > 0) {
        cudaStream_t cs = static_cast<cudaStream_t>(rbsog_stream(s->ctx));
        while ((int)s->ev.size() < 2 * max_steps) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return RBSOG_ECUDA;
            s->ev.push_back(e);
        }
        for (int k = 0; k < max_steps; ++k) {
            cudaEventRecord(s->ev[2 * k], cs);
            st = rbsog_run_async(s->ctx, 1);
            if (st != RBSOG_OK) return st;
            cudaEventRecord(s->ev[2 * k + 1], cs);
        }
        st = rbsog_sync(s->ctx);
        if (st != RBSOG_OK) return st;
        for (int k = 0; k < max_steps; ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, s->ev[2 * k], s->ev[2 * k + 1]);
            s->step_ms.push_back(ms);
            s->gpu_ms += ms;
        }
        // atom-steps actually advanced
        for (int k = 0; k < S; ++k) {
            if (s->slot_ticket[k] < 0) continue;
            const int adv = std::min(s->slot_left[k], max_steps);
            s->atom_steps += (double)s->slot_atoms[k] * adv;
            s->slot_left[k] -= adv;
        }
    }
    if (n_running) *n_running = running;
    if (n_queued) *n_queued = (int)s->queue.size();
    return RBSOG_OK;
}

rbsog_status rbsog_server_result(rbsog_server *s, long long ticket, int *done, double *r, double *v,
                                 rbsog_result *res)
{
    if (!s || !done) return RBSOG_EINVAL;
    auto it = s->req.find(ticket);
    if (it == s->req.end()) return RBSOG_EINVAL;
    const Request &q = it->second;
    *done = q.done ? 1 : 0;
    if (!q.done) return RBSOG_OK;
    if (r) std::memcpy(r, q.r.data(), q.r.size() * sizeof(double));
    if (v) std::memcpy(v, q.v.data(), q.v.size() * sizeof(double));
    if (res) *res = q.res;
    return q.status;
}

rbsog_status rbsog_server_stats(const rbsog_server *s, double *p50_ms, double *p99_ms, double *atom_steps_per_s,
                                long long *steps, int *failed)
{
    if (!s) return RBSOG_EINVAL;
    if (failed) *failed = s->failed;
    std::vector<double> v = s->step_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
        if (v.empty()) return 0.0;
        const size_t i = std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5));
        return v[i];
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (atom_steps_per_s) *atom_steps_per_s = s->gpu_ms > 0 ? s->atom_steps / (s->gpu_ms * 1e-3) : 0.0;
    if (steps) *steps = (long long)s->step_ms.size();
    return RBSOG_OK;
}

}  // extern "C"
