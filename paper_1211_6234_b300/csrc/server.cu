// server.cu -- continuous-batching service for simulation requests.
//
// A request is (L, l, replicas, couplings, sweeps, seed).  Requests share packed
// launches: a pack is one lattice handle whose replica slots belong to different
// requests, each slot carrying its own Philox key, sweep counter and sweep
// budget, so one launch advances many independent chains and each chain is
// bit-identical to the same request run alone.  Packs use the direct path
// (one CTA per slot, as many slots as CTAs fit on the GPU at once) for small
// lattices and the sub-lattice spectral path (or the FFT path) for large ones,
// where all slots share every launch.  Requests too large for a pack get a lone
// handle of their own from a pool.  Packs and lone handles run on separate
// streams, so their work overlaps on the GPU.
//
// mc_server_step() is the whole scheduler and never waits for the GPU:
//   1. retire: a pack or lone handle whose last launch finished credits the
//      sweeps to its requests; finished requests have their observables and
//      spins read back to host memory and give their slots back at once;
//   2. admit: waiting requests, in arrival order, take free slots of a matching
//      pack (or a new pack, or a pooled/new lone handle) while the HBM budget
//      and the active-request limit allow; filling a slot is stream-ordered
//      behind the pack's running launch;
//   3. launch: every idle pack with occupied slots gets its next quantum (each
//      slot min(quantum, remaining) sweeps) and every idle lone handle its next
//      mc_sweep call.
// W~ depends only on (L, image cutoff); it is computed once and copied into
// every handle of that L.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "fft_field.cuh"
#include "internal.cuh"
#include "spectral.cuh"

namespace dipmc {
int lattice_copy_W(mc_lattice *p, const double *W64_dev, int A, int tail);
size_t lattice_footprint(int L, int l, int R);
int lattice_resolved_path(mc_lattice *p);
int pack_enable(mc_lattice *p, int path);
int pack_fill(mc_lattice *p, int slot, int count, uint64_t seed, const RepParams &rp, int init_mode,
              cudaStream_t st);
void pack_set_sweeps(mc_lattice *p, int slot, int count, int nsweeps);
int pack_launch(mc_lattice *p, int measure_every, cudaStream_t st, int *launched);
int pack_group_launch(mc_lattice *const *packs, int count, int measure_every, cudaStream_t st, int *launched);
int pack_group_capacity(mc_lattice *const *packs, int count);
int read_replicas(mc_lattice *p, int first, int count, cudaStream_t st, mc_obs *obs, float *spins);
int lattice_refill(mc_lattice *p, uint64_t seed, const RepParams &rp, int init_mode, cudaStream_t st);
}  // namespace dipmc

using namespace dipmc;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

// Requests that may share a launch: same lattice, spacing, cutoff, proposal and
// measurement interval.
using PackKey = std::tuple<int, int, int, int, double, int>;

// Sites of all slots of a spectral or FFT pack: enough replicas per launch to
// fill the GPU with the contraction's (or the FFT's) blocks.
constexpr long long kPackSites = 1LL << 21;

// Path and slot count of a pack for (L, l), or path -1 if requests of this
// shape run on lone handles.  Small lattices: the direct kernel, one CTA per
// slot; else the sub-lattice spectral path; else the full-lattice FFT.
int pack_shape(int L, int l, int *cap) {
    const long long N = (long long)L * L;
    if (direct_supported(L, l) && L < 128) {
        *cap = std::max(1, direct_resident_ctas(L, l));
        return MC_PATH_DIRECT;
    }
    if (spectral_supported(L, l)) {
        *cap = (int)std::max(1LL, std::min(256LL, kPackSites / N));
        return MC_PATH_SPECTRAL;
    }
    if (fft_supported(L)) {
        *cap = (int)std::max(1LL, std::min(64LL, kPackSites / N));
        return MC_PATH_FFT;
    }
    *cap = 0;
    return -1;
}
// Lone handles are interchangeable when these match.
using SoloKey = std::tuple<int, int, int, int, int, double>;

struct Runner {                 // a handle with its stream and completion event
    mc_lattice *lat = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    size_t bytes = 0;
    bool inflight = false;
};

struct Pack : Runner {
    PackKey key;
    int path = 0;                 // MC_PATH_DIRECT, _SPECTRAL or _FFT
    std::vector<uint64_t> owner;  // per slot: request id, 0 = free
    int measure_every = 0;
};

struct Solo : Runner {
    SoloKey key;
    uint64_t owner = 0;
};

struct Req {
    uint64_t id = 0;
    mc_request r{};
    int state = MC_REQ_QUEUED;
    int64_t done = 0;
    int path = 0;
    Pack *pack = nullptr;
    int slot = -1;
    Solo *solo = nullptr;
    bool packed = false;
    int quantum_sweeps = 0;       // sweeps of this request in its runner's current launch
    double t_submit = 0, t_admit = 0, t_done = 0;
    size_t bytes = 0;
    std::string err;
    std::vector<mc_obs> obs;      // results, after DONE
    std::vector<float> spins;
};

}  // namespace

struct mc_server {
    size_t budget = 0, in_use = 0;
    int max_active = 0, quantum = 0, device = 0, running = 0;
    double max_error = 1e-3;
    uint64_t next_id = 1;
    int64_t completed = 0;
    int64_t grouped_launches = 0;   // launches that carried direct packs of more than one L
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::unique_ptr<Req>> reqs;
    std::map<std::pair<int, int>, double *> wcache;  // (L, A) -> W~ FP64 on the device
    std::vector<std::unique_ptr<Pack>> packs;
    std::vector<std::unique_ptr<Solo>> solos;
};

namespace {

int fail_req(mc_server *s, Req &q, const std::string &why);

int make_runner(Runner &u) {
    if (cudaStreamCreateWithFlags(&u.st, cudaStreamNonBlocking) != cudaSuccess) return MC_ECUDA;
    if (cudaEventCreateWithFlags(&u.ev, cudaEventDisableTiming) != cudaSuccess) return MC_ECUDA;
    return MC_OK;
}

void free_runner(mc_server *s, Runner &u) {
    if (u.st) cudaStreamSynchronize(u.st);
    if (u.lat) mc_destroy(u.lat);
    if (u.ev) cudaEventDestroy(u.ev);
    if (u.st) cudaStreamDestroy(u.st);
    u.lat = nullptr;
    u.ev = nullptr;
    u.st = nullptr;
    s->in_use -= u.bytes;
    u.bytes = 0;
}

int get_W(mc_server *s, int L, int A, const double **out) {
    auto key = std::make_pair(L, A);
    auto it = s->wcache.find(key);
    if (it != s->wcache.end()) {
        *out = it->second;
        return MC_OK;
    }
    mc_lattice *tmp = nullptr;
    int rc = mc_create_lattice(L, L, 1, 1, &tmp);
    if (rc) return rc;
    rc = mc_precompute_W(tmp, A, 1);
    double *W = nullptr;
    std::vector<double> h((size_t)4 * L * L);
    if (!rc) rc = mc_get_W(tmp, h.data());
    mc_destroy(tmp);
    if (!rc && cudaMalloc(&W, sizeof(double) * h.size()) != cudaSuccess) rc = MC_ENOMEM;
    if (!rc && cudaMemcpy(W, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = MC_ECUDA;
    if (rc) {
        cudaFree(W);
        return rc;
    }
    s->wcache[key] = W;
    *out = W;
    return MC_OK;
}

int cutoff_of(const mc_request &r) { return r.image_cutoff > 0 ? r.image_cutoff : 64; }
double cone_of(const mc_request &r) { return r.cone > 0 ? r.cone : 0.5; }

RepParams params_of(const mc_request &r) {
    RepParams p{};
    p.J = (float)r.J;
    p.CD = (float)r.C_D;
    p.K2 = (float)r.K2;
    p.K4 = (float)r.K4;
    p.T = (float)r.T;
    return p;
}

// Free memory held by idle runners until `need` more bytes fit the budget.
bool make_room(mc_server *s, size_t need) {
    if (s->in_use + need <= s->budget) return true;
    for (auto it = s->solos.begin(); it != s->solos.end() && s->in_use + need > s->budget;) {
        Solo &u = **it;
        if (!u.owner && !u.inflight) {
            free_runner(s, u);
            it = s->solos.erase(it);
        } else {
            ++it;
        }
    }
    for (auto it = s->packs.begin(); it != s->packs.end() && s->in_use + need > s->budget;) {
        Pack &u = **it;
        const bool empty = std::all_of(u.owner.begin(), u.owner.end(), [](uint64_t o) { return o == 0; });
        if (empty && !u.inflight) {
            free_runner(s, u);
            it = s->packs.erase(it);
        } else {
            ++it;
        }
    }
    return s->in_use + need <= s->budget;
}

// First run of `count` free consecutive slots, or -1.
int free_run(const Pack &p, int count) {
    int run = 0;
    for (int i = 0; i < (int)p.owner.size(); ++i) {
        run = p.owner[i] ? 0 : run + 1;
        if (run == count) return i - count + 1;
    }
    return -1;
}

// Returns 1 if admitted, 0 if it must wait, <0 if the request failed.
int try_admit(mc_server *s, Req &q) {
    const mc_request &r = q.r;
    const int A = cutoff_of(r);
    int cap = 0;
    const int ppath = pack_shape(r.L, r.l, &cap);
    if (ppath >= 0 && r.replicas <= cap) {
        const PackKey key{r.L, r.l, A, r.proposal, cone_of(r), r.measure_every};
        Pack *pk = nullptr;
        int slot = -1;
        for (auto &p : s->packs)
            if (p->key == key && (slot = free_run(*p, r.replicas)) >= 0) {
                pk = p.get();
                break;
            }
        if (!pk) {
            // a full pack if it fits the budget, else the most slots that do
            if (!make_room(s, lattice_footprint(r.L, r.l, cap))) {
                while (cap > r.replicas && s->in_use + lattice_footprint(r.L, r.l, cap) > s->budget) cap = std::max(r.replicas, cap / 2);
                if (s->in_use + lattice_footprint(r.L, r.l, cap) > s->budget) return 0;
            }
            const size_t bytes = lattice_footprint(r.L, r.l, cap);
            auto np = std::make_unique<Pack>();
            np->key = key;
            np->path = ppath;
            np->measure_every = r.measure_every;
            np->owner.assign(cap, 0);
            const double *W = nullptr;
            int rc = make_runner(*np);
            if (!rc) rc = mc_create_lattice(r.L, r.l, cap, 0, &np->lat);
            if (!rc) rc = mc_set_proposal(np->lat, r.proposal, cone_of(r));
            if (!rc) rc = get_W(s, r.L, A, &W);
            if (!rc) rc = lattice_copy_W(np->lat, W, A, 1);
            if (!rc) rc = pack_enable(np->lat, ppath);
            np->bytes = bytes;
            s->in_use += bytes;
            if (rc) {
                const std::string why = mc_last_error();
                free_runner(s, *np);
                return fail_req(s, q, why);
            }
            pk = np.get();
            slot = 0;
            s->packs.push_back(std::move(np));
        }
        int rc = pack_fill(pk->lat, slot, r.replicas, r.seed, params_of(r), r.init_mode, pk->st);
        if (rc) return fail_req(s, q, mc_last_error());
        for (int i = 0; i < r.replicas; ++i) pk->owner[slot + i] = q.id;
        q.pack = pk;
        q.packed = true;
        q.slot = slot;
        q.path = ppath;
        q.bytes = pk->bytes * r.replicas / pk->owner.size();
    } else {
        const SoloKey key{r.L, r.l, r.replicas, A, r.proposal, cone_of(r)};
        Solo *so = nullptr;
        for (auto &u : s->solos)
            if (!u->owner && !u->inflight && u->key == key) {
                so = u.get();
                break;
            }
        if (!so) {
            const size_t bytes = lattice_footprint(r.L, r.l, r.replicas);
            if (!make_room(s, bytes)) return 0;
            auto nu = std::make_unique<Solo>();
            nu->key = key;
            const double *W = nullptr;
            int rc = make_runner(*nu);
            if (!rc) rc = mc_create_lattice(r.L, r.l, r.replicas, r.seed, &nu->lat);
            if (!rc) rc = mc_set_proposal(nu->lat, r.proposal, cone_of(r));
            if (!rc) rc = get_W(s, r.L, A, &W);
            if (!rc) rc = lattice_copy_W(nu->lat, W, A, 1);
            nu->bytes = bytes;
            s->in_use += bytes;
            if (rc) {
                const std::string why = mc_last_error();
                free_runner(s, *nu);
                return fail_req(s, q, why);
            }
            so = nu.get();
            s->solos.push_back(std::move(nu));
        }
        int rc = lattice_refill(so->lat, r.seed, params_of(r), r.init_mode, so->st);
        if (rc) return fail_req(s, q, mc_last_error());
        so->owner = q.id;
        q.solo = so;
        q.path = lattice_resolved_path(so->lat);
        q.bytes = so->bytes;
    }
    q.state = MC_REQ_RUNNING;
    q.t_admit = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
    ++s->running;
    return 1;
}

void detach(mc_server *s, Req &q) {
    if (q.pack)
        for (int i = 0; i < q.r.replicas; ++i) q.pack->owner[q.slot + i] = 0;
    if (q.solo) q.solo->owner = 0;
    if (q.state == MC_REQ_RUNNING) --s->running;
    q.pack = nullptr;
    q.solo = nullptr;
    q.slot = -1;
    q.bytes = 0;
}

int fail_req(mc_server *s, Req &q, const std::string &why) {
    detach(s, q);
    q.err = why;
    q.state = MC_REQ_FAILED;
    q.t_done = now_s();
    return -1;
}

void finish(mc_server *s, Req &q, mc_lattice *lat, int first, cudaStream_t st) {
    const int R = q.r.replicas;
    q.obs.assign(R, mc_obs{});
    q.spins.assign((size_t)R * 3 * q.r.L * q.r.L, 0.0f);
    const int rc = read_replicas(lat, first, R, st, q.obs.data(), q.spins.data());
    if (rc) {
        fail_req(s, q, mc_last_error());
        return;
    }
    detach(s, q);
    q.state = MC_REQ_DONE;
    q.t_done = now_s();
    ++s->completed;
}

Req *find(mc_server *s, uint64_t id) {
    auto it = s->reqs.find(id);
    return it == s->reqs.end() ? nullptr : it->second.get();
}

// Ids are handed out in sequence and only mc_server_release drops a record, so an id
// below next_id without a record was released.
bool was_released(const mc_server *s, uint64_t id) { return id >= 1 && id < s->next_id && !s->reqs.count(id); }

// Credit a finished launch to the requests it carried.
void retire(mc_server *s, Runner &u, bool is_pack) {
    if (!u.inflight) return;
    const cudaError_t e = cudaEventQuery(u.ev);
    if (e == cudaErrorNotReady) return;
    u.inflight = false;
    std::vector<uint64_t> ids;
    if (is_pack) {
        for (uint64_t o : static_cast<Pack &>(u).owner)
            if (o && (ids.empty() || ids.back() != o)) ids.push_back(o);
    } else if (static_cast<Solo &>(u).owner) {
        ids.push_back(static_cast<Solo &>(u).owner);
    }
    for (uint64_t id : ids) {
        Req *q = find(s, id);
        if (!q || q->state != MC_REQ_RUNNING) continue;
        if (e != cudaSuccess) {
            fail_req(s, *q, cudaGetErrorString(e));
            continue;
        }
        q->done += q->quantum_sweeps;
        q->quantum_sweeps = 0;
        if (q->done >= q->r.sweeps) finish(s, *q, u.lat, is_pack ? q->slot : 0, u.st);
    }
}

// The next quantum of every occupied slot of an idle pack (pack_set_sweeps);
// returns the number of slots with sweeps to run.
int plan_pack(mc_server *s, Pack &p) {
    if (p.inflight) return 0;
    int active = 0;
    for (int i = 0; i < (int)p.owner.size();) {
        Req *q = p.owner[i] ? find(s, p.owner[i]) : nullptr;
        if (!q) {
            ++i;
            continue;
        }
        const int n = (int)std::min<int64_t>(s->quantum, q->r.sweeps - q->done);
        pack_set_sweeps(p.lat, i, q->r.replicas, n);
        q->quantum_sweeps = n;
        if (n > 0) active += q->r.replicas;
        i += q->r.replicas;
    }
    return active;
}

void fail_pack(mc_server *s, Pack &p, const std::string &why) {
    for (uint64_t o : p.owner) {
        Req *q = o ? find(s, o) : nullptr;
        if (q && q->state == MC_REQ_RUNNING) fail_req(s, *q, why);
    }
}

void launch_pack(mc_server *s, Pack &p) {
    if (p.inflight || plan_pack(s, p) == 0) return;
    int launched = 0;
    int rc = pack_launch(p.lat, p.measure_every, p.st, &launched);
    if (!rc && cudaEventRecord(p.ev, p.st) != cudaSuccess) rc = MC_ECUDA;
    if (rc) {
        fail_pack(s, p, mc_last_error());
        return;
    }
    p.inflight = launched > 0;
}

// Idle direct packs of one (C, proposal, cone, measurement interval) whose slots
// with work all fit one resident wave of a grouped launch run as ONE launch on
// the first pack's stream (lattices of different L side by side); the other packs'
// streams are joined to it by events before and after, so their fills and
// read-backs stay ordered.  Larger groups run pack by pack, at each pack's own
// launch shape (a grouped launch takes the largest lattice's shape for every CTA).
void launch_groups(mc_server *s) {
    std::map<std::tuple<int, int, double, int>, std::vector<Pack *>> groups;
    for (auto &p : s->packs) {
        if (p->inflight || p->path != MC_PATH_DIRECT) continue;
        const int L = std::get<0>(p->key), l = std::get<1>(p->key);
        groups[std::make_tuple(L / l, std::get<3>(p->key), std::get<4>(p->key), p->measure_every)].push_back(p.get());
    }
    for (auto &kv : groups) {
        std::vector<Pack *> &ps = kv.second;
        if (ps.size() < 2) continue;
        std::vector<Pack *> live;
        int active = 0;
        for (Pack *p : ps) {
            const int a = plan_pack(s, *p);
            if (a > 0) {
                live.push_back(p);
                active += a;
            }
        }
        bool mixed = false;
        for (Pack *p : live) mixed = mixed || std::get<0>(p->key) != std::get<0>(live[0]->key);
        if (live.size() < 2 || !mixed) continue;   // launched one by one below
        std::vector<mc_lattice *> lats;
        for (Pack *p : live) lats.push_back(p->lat);
        if (active > pack_group_capacity(lats.data(), (int)lats.size())) continue;
        Pack &h = *live[0];
        int rc = MC_OK;
        for (size_t i = 1; i < live.size() && !rc; ++i) {
            if (cudaEventRecord(live[i]->ev, live[i]->st) != cudaSuccess ||
                cudaStreamWaitEvent(h.st, live[i]->ev, 0) != cudaSuccess)
                rc = MC_ECUDA;
        }
        int launched = 0;
        if (!rc) rc = pack_group_launch(lats.data(), (int)lats.size(), h.measure_every, h.st, &launched);
        if (!rc && cudaEventRecord(h.ev, h.st) != cudaSuccess) rc = MC_ECUDA;
        for (size_t i = 1; i < live.size() && !rc; ++i) {
            if (cudaStreamWaitEvent(live[i]->st, h.ev, 0) != cudaSuccess ||
                cudaEventRecord(live[i]->ev, live[i]->st) != cudaSuccess)
                rc = MC_ECUDA;
        }
        if (rc) {
            const std::string why = mc_last_error();
            for (Pack *p : live) fail_pack(s, *p, why);
            continue;
        }
        for (Pack *p : live) p->inflight = launched > 0;
        ++s->grouped_launches;
    }
}

void launch_solo(mc_server *s, Solo &u) {
    if (u.inflight || !u.owner) return;
    Req *q = find(s, u.owner);
    if (!q) return;
    const int n = (int)std::min<int64_t>(s->quantum, q->r.sweeps - q->done);
    if (n <= 0) return;
    int rc = mc_sweep(u.lat, n, q->r.measure_every, u.st);
    if (!rc && cudaEventRecord(u.ev, u.st) != cudaSuccess) rc = MC_ECUDA;
    if (rc) {
        fail_req(s, *q, mc_last_error());
        return;
    }
    q->quantum_sweeps = n;
    u.inflight = true;
}

}  // namespace

extern "C" {

int mc_footprint(int L, int l, int replicas, size_t *bytes) {
    if (!bytes) return set_last_error(MC_EINVAL, "bytes is null");
    if (L < 2 || L > 4096 || l < 2 || l > L || L % l || replicas < 1)
        return set_last_error(MC_EINVAL, "mc_footprint needs 2 <= l <= L <= 4096, L % l == 0, replicas >= 1");
    *bytes = lattice_footprint(L, l, replicas);
    return MC_OK;
}

int mc_server_create(size_t hbm_budget_bytes, int max_active, int quantum_sweeps, double max_error,
                     mc_server **out) {
    if (!out) return set_last_error(MC_EINVAL, "out is null");
    *out = nullptr;
    if (hbm_budget_bytes == 0 || max_active < 1 || quantum_sweeps < 1 || !(max_error > 0))
        return set_last_error(MC_EINVAL, "mc_server_create: budget, max_active, quantum and max_error must be positive");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_last_error(MC_ECUDA, "cudaGetDevice failed");
    mc_server *s = new mc_server();
    s->budget = hbm_budget_bytes;
    s->max_active = max_active;
    s->quantum = quantum_sweeps;
    s->max_error = max_error;
    s->device = dev;
    *out = s;
    return MC_OK;
}

int mc_server_submit(mc_server *s, const mc_request *r, uint64_t *id) {
    if (!s || !r || !id) return set_last_error(MC_EINVAL, "null argument");
    mc_request q = *r;
    if (q.replicas < 1) q.replicas = 1;
    if (q.L < 2 || q.L > 4096 || q.sweeps < 0 || !(q.T > 0) || q.measure_every < 0 || q.init_mode < 0 ||
        q.init_mode > 3 || q.init_mode == 2 || q.proposal < 0 || q.proposal > 2)
        return set_last_error(MC_EINVAL, "request needs 2 <= L <= 4096, T > 0, sweeps >= 0, measure_every >= 0, "
                                         "init_mode in {0, 1, 3} and proposal in {0, 1, 2}");
    if (q.l == 0) {
        // the smallest spacing within the error bound; a larger divisor of L only
        // lowers the error, so move up to the first one the direct pack serves (measured
        // at L = 96: the direct kernel at l = 24 runs 64 packed requests several times
        // faster than the spectral pack at l = 16), else to the first any pack serves
        int rc = mc_choose_spacing(q.L, q.C_D, q.T, s->max_error, &q.l);
        if (rc) return rc;
        int cap = 0, best = -1;
        for (int d = q.l; d <= q.L && best < 0; ++d)
            if (q.L % d == 0 && pack_shape(q.L, d, &cap) == MC_PATH_DIRECT) best = d;
        for (int d = q.l; d <= q.L && best < 0; ++d)
            if (q.L % d == 0 && pack_shape(q.L, d, &cap) >= 0) best = d;
        if (best > 0) q.l = best;
    }
    if (q.l < 2 || q.l > q.L || q.L % q.l) return set_last_error(MC_EINVAL, "request needs 2 <= l <= L and L % l == 0");
    if (lattice_footprint(q.L, q.l, q.replicas) > s->budget)
        return set_last_error(MC_ENOMEM, "request footprint exceeds the server's HBM budget");
    auto rq = std::make_unique<Req>();
    rq->id = s->next_id++;
    rq->r = q;
    rq->t_submit = now_s();
    *id = rq->id;
    s->queue.push_back(rq->id);
    s->reqs[rq->id] = std::move(rq);
    return MC_OK;
}

int mc_server_step(mc_server *s) {
    if (!s) return set_last_error(MC_EINVAL, "null server");
    if (cudaSetDevice(s->device) != cudaSuccess) return set_last_error(MC_ECUDA, "cudaSetDevice failed");
    for (auto &p : s->packs) retire(s, *p, true);
    for (auto &u : s->solos) retire(s, *u, false);
    while (!s->queue.empty()) {
        Req *q = find(s, s->queue.front());
        if (!q || q->state != MC_REQ_QUEUED) {
            s->queue.pop_front();
            continue;
        }
        if (s->running >= s->max_active) break;
        if (try_admit(s, *q) == 0) break;  // the first in line waits for memory: arrival order is kept
        s->queue.pop_front();
    }
    // requests of zero sweeps finish at admission
    for (auto &kv : s->reqs) {
        Req &q = *kv.second;
        if (q.state == MC_REQ_RUNNING && q.r.sweeps == 0) {
            if (q.pack) finish(s, q, q.pack->lat, q.slot, q.pack->st);
            else if (q.solo) finish(s, q, q.solo->lat, 0, q.solo->st);
        }
    }
    launch_groups(s);
    for (auto &p : s->packs) launch_pack(s, *p);
    for (auto &u : s->solos) launch_solo(s, *u);
    return MC_OK;
}

int mc_server_poll(mc_server *s, uint64_t id, int *state, int64_t *sweeps_done) {
    if (!s) return set_last_error(MC_EINVAL, "null server");
    Req *q = find(s, id);
    if (!q && was_released(s, id)) {
        if (state) *state = MC_REQ_RELEASED;
        if (sweeps_done) *sweeps_done = 0;
        return MC_OK;
    }
    if (!q) return set_last_error(MC_EINVAL, "unknown request id");
    if (state) *state = q->state;
    if (sweeps_done) *sweeps_done = q->done;
    return MC_OK;
}

int mc_server_request_info(mc_server *s, uint64_t id, mc_request_info *out) {
    if (!s || !out) return set_last_error(MC_EINVAL, "null argument");
    Req *q = find(s, id);
    if (!q && was_released(s, id)) {
        std::memset(out, 0, sizeof *out);
        out->state = MC_REQ_RELEASED;
        return MC_OK;
    }
    if (!q) return set_last_error(MC_EINVAL, "unknown request id");
    std::memset(out, 0, sizeof *out);
    out->state = q->state;
    out->sweeps_done = q->done;
    out->l = q->r.l;
    out->path = q->path;
    out->packed = q->packed ? 1 : 0;
    out->t_submit = q->t_submit;
    out->t_admit = q->t_admit;
    out->t_done = q->t_done;
    out->bytes = q->bytes;
    std::strncpy(out->error, q->err.c_str(), sizeof(out->error) - 1);
    return MC_OK;
}

int mc_server_collect(mc_server *s, uint64_t id, int replica, mc_obs *out) {
    if (!s || !out) return set_last_error(MC_EINVAL, "null argument");
    Req *q = find(s, id);
    if (!q && was_released(s, id)) return set_last_error(MC_ENOTREADY, "request was released");
    if (!q) return set_last_error(MC_EINVAL, "unknown request id");
    if (q->state != MC_REQ_DONE) return set_last_error(MC_ENOTREADY, "request is not done");
    if (replica < 0 || replica >= q->r.replicas) return set_last_error(MC_EINVAL, "replica out of range");
    *out = q->obs[replica];
    return MC_OK;
}

int mc_server_get_spins(mc_server *s, uint64_t id, float *dst_host) {
    if (!s || !dst_host) return set_last_error(MC_EINVAL, "null argument");
    Req *q = find(s, id);
    if (!q && was_released(s, id)) return set_last_error(MC_ENOTREADY, "request was released");
    if (!q) return set_last_error(MC_EINVAL, "unknown request id");
    if (q->state != MC_REQ_DONE) return set_last_error(MC_ENOTREADY, "request is not done");
    std::memcpy(dst_host, q->spins.data(), sizeof(float) * q->spins.size());
    return MC_OK;
}

int mc_server_release(mc_server *s, uint64_t id) {
    if (!s) return set_last_error(MC_EINVAL, "null server");
    Req *q = find(s, id);
    if (!q && was_released(s, id)) return MC_OK;
    if (!q) return set_last_error(MC_EINVAL, "unknown request id");
    if (q->state == MC_REQ_RUNNING) {
        // A pack's launch that still carries the request runs on untouched; the
        // freed slots are refilled only behind it, in stream order.  A lone
        // handle is waited for before it can go back to the pool.
        if (q->solo && q->solo->inflight) {
            cudaStreamSynchronize(q->solo->st);
            q->solo->inflight = false;
        }
        detach(s, *q);
    }
    // the record goes too, so a long-lived server does not grow with the requests it
    // has served; the id still polls as released (a queued id is skipped at admission)
    s->reqs.erase(id);
    return MC_OK;
}

int mc_server_get_stats(mc_server *s, mc_server_stats *out) {
    if (!s || !out) return set_last_error(MC_EINVAL, "null argument");
    std::memset(out, 0, sizeof *out);
    for (auto &kv : s->reqs) {
        const int st = kv.second->state;
        if (st == MC_REQ_QUEUED) ++out->queued;
        else if (st == MC_REQ_RUNNING) ++out->running;
        else if (st == MC_REQ_DONE) ++out->done;
        else if (st == MC_REQ_FAILED) ++out->failed;
    }
    out->completed = s->completed;
    out->grouped_launches = s->grouped_launches;
    out->bytes_in_use = s->in_use;
    out->budget = s->budget;
    out->packs = (int)s->packs.size();
    out->lone = (int)s->solos.size();
    return MC_OK;
}

int mc_server_destroy(mc_server *s) {
    if (!s) return MC_OK;
    cudaSetDevice(s->device);
    for (auto &p : s->packs) free_runner(s, *p);
    for (auto &u : s->solos) free_runner(s, *u);
    for (auto &kv : s->wcache) cudaFree(kv.second);
    delete s;
    return MC_OK;
}

}  // extern "C"
