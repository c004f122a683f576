// api.cu -- the C ABI of libdipmc (declared in include/dipmc.h): handle
// lifetime, argument validation, device buffers and dispatch to the kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "fft_cluster.cuh"
#include "fft_field.cuh"
#include "incremental.cuh"
#include "internal.cuh"
#include "spectral.cuh"
#include "tc_field.cuh"
#include "window.cuh"

using namespace dipmc;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(MC_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);   \
    } while (0)

constexpr uint32_t kMagic = 0x444d4331u;  // "DMC1"
constexpr int kVersion = 2;

}  // namespace

int dipmc::set_last_error(int code, const char *msg) {
    g_err = msg;
    return code;
}

struct mc_lattice {
    int L = 0, l = 0, R = 0, device = 0;
    uint64_t seed = 0;
    int proposal = 0;
    double cone = 0.5;
    int schedule = 0;
    int path = MC_PATH_AUTO;
    int threads_hint = 512;
    std::vector<RepParams> hp;
    RepParams *dparams = nullptr;
    float *spins = nullptr;   // [R][3][N]
    float *field = nullptr;   // [R][3][N] scratch for full-field evaluations
    double *W64 = nullptr;    // [4][N]
    float *W32 = nullptr;     // [4][N]
    double *energy = nullptr; // [R] tracked energy
    double *etmp = nullptr;   // [R] scratch for mc_energy
    ObsAcc *obs = nullptr;    // [R]
    double *theta2 = nullptr; // [R][N]
    double *eta_dev = nullptr; // [R] eta of the last read-back
    // pinned staging of the observables read-back: [cap] accumulators, then [cap]
    // energies and [cap] eta values (grown on demand, kept for the handle's life)
    unsigned char *obs_pin = nullptr;
    int obs_pin_cap = 0;
    uint64_t t = 0;
    bool W_ready = false, energy_valid = false;
    int A = 0, tail = 0;
    cudaStream_t last = nullptr;
    // windowed / tensor-core paths
    int window_B = 0;
    int tc_kblocks = 0, tc_ntile = 0, steps_layout = 0;   // launch shapes (mc_tuning)
    int plan_kb = 0, plan_nt = 0;                         // shapes the current tensor plan was made with
    __nv_bfloat16 *spins_hi = nullptr, *spins_lo = nullptr, *wsh = nullptr;
    TcUnit *units = nullptr;
    int nunits = 0, NT = 0, tmem_cols = 0, plan_Sw = 0;
    float *tcpart = nullptr;      // [nunits][NT][128] partial tiles of the split-K contraction
    alignas(64) unsigned char tm_hi[128], tm_lo[128];   // TMA maps of spins_hi / spins_lo
    int tm_NT = 0;
    int *tile_first = nullptr;    // [ntiles * mtiles + 1]
    int mtiles = 0, ntiles = 0;
    int *err_flag = nullptr;
    bool wsh_ready = false;
    bool wsh_spec2 = false;     // wsh holds the signed cell-grid spectra of W~
    float4 *wq = nullptr;     // W~ tables of the windowed paths (wq_table_elems)
    float *What = nullptr;    // [4][N] transform of W~ (FFT path), transposed layout
    float2 *fft_scratch = nullptr;
    bool what_ready = false;
    // cluster-resident transform path: W^ on the half plane, the spins' transform and row scratch
    float *cl_What = nullptr;
    float2 *cl_S = nullptr, *cl_rows = nullptr;
    bool cl_ready = false;
    // sub-lattice spectral path
    float2 *specT = nullptr, *specS = nullptr, *specH = nullptr;
    int *specOff = nullptr;
    bool spec_ready = false;
    int spec_esplit = 0;
    // CUDA graphs of the multi-launch paths, keyed by (path, nsweeps, measure_every)
    uint32_t *t_dev = nullptr;            // sweep counter at the start of the current call
    cudaStream_t own = nullptr;           // capture/replay stream (joined to the caller's by events)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;
    std::map<std::tuple<int, int, int>, int> seen;
    // kernel timing (events recorded around launches while enabled)
    bool timing = false;
    unsigned long long *wcyc = nullptr;   // [4] sub-step kernel cycle counters while timing
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> tev[MC_NKCLASS];
    // energy histogram of the measured sweeps, [R][hist_bins]
    unsigned long long *hist = nullptr;
    double hist_lo = 0.0, hist_scale = 0.0;
    int hist_bins = 0;
    // grouped direct launches (mc_sweep_group, server): descriptors staged through
    // pinned memory, one copy in flight at a time
    SlotGeom *geom_dev = nullptr, *geom_pin = nullptr;
    int geom_cap = 0;
    cudaEvent_t geom_copied = nullptr;
    // packed launches (serving): per-slot stream state, host shadow and pinned staging
    bool packed = false;
    SlotState *slots_dev = nullptr, *slots_pin = nullptr;
    RepParams *params_pin = nullptr;
    std::vector<SlotState> slots_host;
    cudaEvent_t slots_copied = nullptr;

    int N() const { return L * L; }
    int n() const { return (L / l) * (L / l); }
    size_t spin_floats() const { return (size_t)R * 3 * N(); }
};

namespace {

void free_all(mc_lattice *p) {
    cudaFree(p->geom_dev);
    cudaFreeHost(p->geom_pin);
    if (p->geom_copied) cudaEventDestroy(p->geom_copied);
    cudaFree(p->dparams);
    cudaFree(p->spins);
    cudaFree(p->field);
    cudaFree(p->W64);
    cudaFree(p->W32);
    cudaFree(p->energy);
    cudaFree(p->etmp);
    cudaFree(p->obs);
    cudaFree(p->theta2);
    cudaFree(p->eta_dev);
    if (p->obs_pin) cudaFreeHost(p->obs_pin);
    cudaFree(p->spins_hi);
    cudaFree(p->spins_lo);
    cudaFree(p->wsh);
    cudaFree(p->units);
    cudaFree(p->tcpart);
    cudaFree(p->tile_first);
    cudaFree(p->err_flag);
    cudaFree(p->wq);
    cudaFree(p->What);
    cudaFree(p->fft_scratch);
    cudaFree(p->cl_What);
    cudaFree(p->cl_S);
    cudaFree(p->cl_rows);
    cudaFree(p->t_dev);
    cudaFree(p->wcyc);
    for (auto &g : p->graphs) cudaGraphExecDestroy(g.second);
    p->graphs.clear();
    if (p->own) cudaStreamDestroy(p->own);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    cudaFree(p->hist);
    cudaFree(p->specT);
    cudaFree(p->specS);
    cudaFree(p->specH);
    cudaFree(p->specOff);
    cudaFree(p->slots_dev);
    if (p->slots_pin) cudaFreeHost(p->slots_pin);
    if (p->params_pin) cudaFreeHost(p->params_pin);
    if (p->slots_copied) cudaEventDestroy(p->slots_copied);
}

void drop_graphs(mc_lattice *p) {
    for (auto &g : p->graphs) cudaGraphExecDestroy(g.second);
    p->graphs.clear();
    p->seen.clear();
}

// Records an event pair around a launch when timing is on.
struct TimedLaunch {
    mc_lattice *p;
    int cls;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    TimedLaunch(mc_lattice *p_, int cls_, cudaStream_t st_) : p(p_), cls(cls_), st(st_) {
        if (p->timing && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
            cudaEventRecord(a, st);
    }
    ~TimedLaunch() {
        if (a && b) {
            cudaEventRecord(b, st);
            p->tev[cls].push_back({a, b});
        } else if (a) {
            cudaEventDestroy(a);   // the second event could not be created
        }
    }
};

void clear_timing(mc_lattice *p) {
    for (auto &v : p->tev) {
        for (auto &e : v) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
        v.clear();
    }
}

// Sub-steps per window: the given B, else the largest power of two dividing l^2
// with B*n <= 512 (tensor path: a multiple of 128, and <= 256 unless the cell-grid
// spectra serve 512 sites with two sub-step CTAs per SM).  The in-window pushes grow
// with B*n per site while the per-window costs shrink; at L = 64, l = 32 the tensor
// path is fastest with 512-site windows (50.7 against 53.5 ms per 100 sweeps of
// 256 replicas).
int window_of(const mc_lattice *p, bool tensor) {
    const int ll = p->l * p->l, n = p->n();
    if (p->window_B > 0) return p->window_B;
    const int cap = (!tensor || (tc_spec2_supported(p->L, p->l, 512) &&
                                 window_smem_bytes(p->L, 512, n) <= kWindowSmemTwoCtas)) ? 512 : 256;
    int best = 0;
    for (int B = 1; B <= ll; B <<= 1) {
        if (ll % B) continue;
        if (B * n > cap) break;
        if (tensor && (B * n) % 128) continue;
        best = B;
    }
    return best;
}

bool path_supported(const mc_lattice *p, int path) {
    switch (path) {
        case MC_PATH_DIRECT: return direct_supported(p->L, p->l);
        case MC_PATH_WINDOW_F32: {
            const int B = window_of(p, false);
            return B > 0 && window_supported(p->L, p->l, B);
        }
        case MC_PATH_TENSOR: {
            const int B = window_of(p, true);
            return B > 0 && tc_supported(p->L, p->l, B) && window_supported(p->L, p->l, B);
        }
        case MC_PATH_FFT: return fft_supported(p->L);
        case MC_PATH_SPECTRAL: return spectral_supported(p->L, p->l);
        case MC_PATH_INCREMENTAL: return incremental_supported(p->L, p->l);
        case MC_PATH_FFT_CLUSTER: return cluster_supported(p->L, p->l);
        default: return false;
    }
}

EnergyHist hist_of(const mc_lattice *p) {
    EnergyHist h;
    if (p->hist && p->hist_bins > 0) {
        h.counts = p->hist;
        h.lo = p->hist_lo;
        h.scale = p->hist_scale;
        h.nbins = p->hist_bins;
    }
    return h;
}

int resolve_path(const mc_lattice *p) {
    if (p->path != MC_PATH_AUTO) return p->path;
    // measured at L = 64: the tensor path is 3-4x the direct path from 16 replicas up
    // (and 11x for l = L), so it leads wherever its window fits
    if (path_supported(p, MC_PATH_TENSOR)) return MC_PATH_TENSOR;
    if (direct_supported(p->L, p->l)) return MC_PATH_DIRECT;
    if (spectral_supported(p->L, p->l)) return MC_PATH_SPECTRAL;
    if (fft_supported(p->L)) return MC_PATH_FFT;
    if (path_supported(p, MC_PATH_WINDOW_F32)) return MC_PATH_WINDOW_F32;
    return -1;
}

int upload_params(mc_lattice *p) {
    CK(cudaMemcpy(p->dparams, p->hp.data(), sizeof(RepParams) * p->R, cudaMemcpyHostToDevice));
    return MC_OK;
}

int clear_obs(mc_lattice *p, cudaStream_t st) {
    CK(cudaMemsetAsync(p->obs, 0, sizeof(ObsAcc) * p->R, st));
    CK(cudaMemsetAsync(p->theta2, 0, sizeof(double) * (size_t)p->R * p->N(), st));
    if (p->hist) CK(cudaMemsetAsync(p->hist, 0, sizeof(unsigned long long) * p->R * p->hist_bins, st));
    return MC_OK;
}

uint2 key_of(uint64_t seed) { return make_uint2((uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)); }

int full_field(mc_lattice *p, cudaStream_t st);

int ensure_fft(mc_lattice *p, cudaStream_t st);

// Energy anchor of replicas [first, first + count): their full field by the
// O(N log N) transform for power-of-two L >= 64 (a 256-replica L = 64 anchor:
// tens of microseconds instead of milliseconds for the O(N^2) sum), else by the
// direct sum; then the energy sums.  Both are per replica, so an anchor does not
// depend on which other replicas share the handle.
int anchor_replicas(mc_lattice *p, int first, int count, cudaStream_t st) {
    const size_t off = (size_t)first * 3 * p->N();
    cudaError_t e;
    if (fft_supported(p->L) && p->L >= 64) {
        int rc = ensure_fft(p, st);
        if (rc) return rc;
        TimedLaunch tl(p, MC_K_FULL_FIELD, st);
        e = launch_fft_field(p->L, count, p->spins + off, p->What, p->fft_scratch, p->field + off, st);
    } else {
        TimedLaunch tl(p, MC_K_FULL_FIELD, st);
        e = launch_full_field(p->L, count, p->W32, p->spins + off, p->field + off, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "full-field evaluation");
    e = launch_energy(p->L, count, p->spins + off, p->field + off, p->dparams + first, p->energy + first, st);
    if (e != cudaSuccess) return cuda_fail(e, "energy kernel");
    return MC_OK;
}

int anchor_energy(mc_lattice *p, cudaStream_t st) {
    int rc = anchor_replicas(p, 0, p->R, st);
    if (rc) return rc;
    p->energy_valid = true;
    return MC_OK;
}

int check(mc_lattice *p) {
    if (!p) return fail(MC_EINVAL, "null lattice handle");
    CK(cudaSetDevice(p->device));
    return MC_OK;
}

// A bounded device wait that gave up leaves a flag; report it at the next sync point.
int check_device_flag(mc_lattice *p) {
    if (!p->err_flag) return MC_OK;
    int v = 0;
    CK(cudaMemcpy(&v, p->err_flag, sizeof v, cudaMemcpyDeviceToHost));
    if (v) {
        cudaMemset(p->err_flag, 0, sizeof v);
        if (v == 2) return fail(MC_ECUDA, "tensor-core field: shared-memory stages not 1024-byte aligned; results invalid");
        if (v == 3) return fail(MC_ETIMEOUT, "sub-step kernel: the bulk copy of the spins did not complete; results of the last sweep are invalid");
        return fail(MC_ETIMEOUT, "a tensor-core pipeline wait timed out; results of the last sweep are invalid");
    }
    return MC_OK;
}

#define CKA(call)                                                        \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);              \
    } while (0)

int ensure_tensor_buffers(mc_lattice *p, int Sw, cudaStream_t st) {
    const size_t N = p->N(), R = p->R;
    if (!p->spins_hi) {
        CKA(cudaMalloc(&p->spins_hi, sizeof(__nv_bfloat16) * 3 * N * R));
        CKA(cudaMalloc(&p->spins_lo, sizeof(__nv_bfloat16) * 3 * N * R));
        CKA(cudaMalloc(&p->err_flag, sizeof(int)));
        CKA(cudaMemset(p->err_flag, 0, sizeof(int)));
    }
    // operand tables: the Toeplitz copies of W~, or for L = 2l with a 256- or 512-site window the
    // signed spectra of W~ over the 2 x 2 cell grid (the lattice keeps one kind)
    const bool spec2 = tc_spec2_supported(p->L, p->l, Sw);
    if (!p->wsh) CKA(cudaMalloc(&p->wsh, sizeof(__nv_bfloat16) * std::max(tc_wsh_elems(p->L), tc_t2_elems(p->l))));
    if (!p->wsh_ready || p->wsh_spec2 != spec2) {
        cudaError_t e = spec2 ? launch_build_t2(p->L, p->W64, p->wsh, st) : launch_build_wsh(p->L, p->W64, p->wsh, st);
        if (e != cudaSuccess) return cuda_fail(e, "W~ bf16 tables");
        p->wsh_ready = true;
        p->wsh_spec2 = spec2;
    }
    if (p->plan_Sw != Sw || p->plan_kb != p->tc_kblocks || p->plan_nt != p->tc_ntile) {
        cudaFree(p->units);
        cudaFree(p->tcpart);
        cudaFree(p->tile_first);
        p->units = nullptr; p->tcpart = nullptr; p->tile_first = nullptr;
        int dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        std::vector<TcUnit> u(65536);
        std::vector<int> tf(1 << 16);
        const int nu = tc_plan(p->L, Sw, p->R, nsm, u.data(), (int)u.size(), &p->NT, &p->tmem_cols, tf.data(),
                               &p->mtiles, &p->ntiles, spec2, p->tc_kblocks, p->tc_ntile);
        if (nu <= 0) return fail(MC_EINVAL, "tensor-core plan failed for Sw=%d R=%d", Sw, p->R);
        CKA(cudaMalloc(&p->units, sizeof(TcUnit) * nu));
        CKA(cudaMemcpy(p->units, u.data(), sizeof(TcUnit) * nu, cudaMemcpyHostToDevice));
        const int ntf = p->ntiles * p->mtiles + 1;
        CKA(cudaMalloc(&p->tile_first, sizeof(int) * ntf));
        CKA(cudaMemcpy(p->tile_first, tf.data(), sizeof(int) * ntf, cudaMemcpyHostToDevice));
        CKA(cudaMalloc(&p->tcpart, sizeof(float) * (size_t)nu * p->NT * 128));
        p->nunits = nu;
        p->plan_Sw = Sw;
        p->plan_kb = p->tc_kblocks;
        p->plan_nt = p->tc_ntile;
        if (tc_map_bytes() > sizeof(p->tm_hi) || tc_encode_map(p->tm_hi, p->spins_hi, p->L, p->R, p->NT) ||
            tc_encode_map(p->tm_lo, p->spins_lo, p->L, p->R, p->NT))
            return fail(MC_ECUDA, "TMA map of the bf16 spins could not be encoded");
        p->tm_NT = p->NT;
    }
    return MC_OK;
}

int run_windows(mc_lattice *p, int path, int nsweeps, int measure_every, float *trace, cudaStream_t st) {
    const bool tensor = path == MC_PATH_TENSOR;
    const int B = window_of(p, tensor);
    const int ll = p->l * p->l, n = p->n(), Sw = B * n, nwin = ll / B;
    const bool spec2 = tensor && tc_spec2_supported(p->L, p->l, Sw);
    if (tensor) {
        int rc = ensure_tensor_buffers(p, Sw, st);
        if (rc) return rc;
        // the B operand: bf16 hi/lo of the spins, or of their cell-grid spectra
        cudaError_t e = spec2 ? launch_spec2_init(p->L, p->R, p->spins, p->spins_hi, p->spins_lo, st)
                              : launch_spins_to_bf16((size_t)p->R * 3 * p->N(), p->spins, p->spins_hi, p->spins_lo, st);
        if (e != cudaSuccess) return cuda_fail(e, "bf16 operand of the spins");
    }
    WindowConfig c{};
    c.t_dev = p->t_dev;
    c.L = p->L; c.l = p->l; c.R = p->R;
    c.key = key_of(p->seed);
    c.nsweeps_call = nsweeps;
    c.B = B;
    c.proposal = p->proposal;
    c.cap_c1 = (float)(1.0 - std::cos(p->cone));
    c.schedule = p->schedule;
    c.stale_mode = tensor ? (spec2 ? 3 : 2) : 0;   // tensor path: the sub-step kernel sums the split-K partial tiles
    c.NT = p->NT;
    c.mtiles = p->mtiles;
    c.layout = p->steps_layout;
    {
        int dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        c.nsm = nsm;
    }
    WindowBuffers b{};
    b.W32 = p->W32; b.spins = p->spins;
    b.spins_hi = tensor ? p->spins_hi : nullptr;
    b.spins_lo = tensor ? p->spins_lo : nullptr;
    b.params = p->dparams; b.energy = p->energy; b.obs = p->obs; b.theta2 = p->theta2;
    b.trace = trace;
    b.stale = tensor ? nullptr : p->field;
    b.part = tensor ? p->tcpart : nullptr;
    b.tile_first = tensor ? p->tile_first : nullptr;
    b.wq = p->wq;
    b.hist = hist_of(p);
    b.cycles = p->timing ? p->wcyc : nullptr;
    b.error = tensor ? p->err_flag : nullptr;
    TcFieldArgs ta{};
    if (tensor) {
        ta.L = p->L; ta.Sw = Sw; ta.R = p->R; ta.NT = p->NT; ta.tmem_cols = p->tmem_cols;
        ta.units = p->units; ta.wsh = p->wsh;
        ta.l = p->l; ta.schedule = p->schedule; ta.key = c.key; ta.t_dev = p->t_dev;
        ta.spec2 = spec2 ? 1 : 0;
        ta.spins_hi = p->spins_hi; ta.spins_lo = p->spins_lo; ta.error = p->err_flag;
        ta.part = p->tcpart; ta.tile_first = p->tile_first; ta.mtiles = p->mtiles; ta.ntiles = p->ntiles;
    }
    for (int it = 0; it < nsweeps; ++it) {
        c.t = (uint32_t)(p->t + (uint64_t)it);
        c.it = it;
        for (int w = 0; w < nwin; ++w) {
            cudaError_t e;
            if (tensor) {
                ta.t_host = c.t;
                ta.it = it;
                ta.k0 = w * B;
                {
                    TimedLaunch tl(p, MC_K_TC_FIELD, st);
                    e = launch_tc_field(ta, p->nunits, p->tm_hi, p->tm_lo, st);
                }
                if (e != cudaSuccess) return cuda_fail(e, "tensor-core field launch");
            } else {
                TimedLaunch tl(p, MC_K_FULL_FIELD, st);
                e = launch_full_field(p->L, p->R, p->W32, p->spins, p->field, st);
                if (e != cudaSuccess) return cuda_fail(e, "full-field kernel");
            }
            c.w = w;
            c.measure = (measure_every > 0 && ((it + 1) % measure_every) == 0 && w == nwin - 1) ? 1 : 0;
            {
                TimedLaunch tl(p, MC_K_WINDOW_STEPS, st);
                e = launch_window_steps(c, b, st);
            }
            if (e != cudaSuccess) return cuda_fail(e, "window step kernel launch");
        }
    }
    return MC_OK;
}

int ensure_fft(mc_lattice *p, cudaStream_t st) {
    if (!p->What) CKA(cudaMalloc(&p->What, sizeof(float) * 4 * (size_t)p->N()));
    if (!p->fft_scratch) CKA(cudaMalloc(&p->fft_scratch, fft_scratch_bytes(p->L, p->R)));
    if (!p->what_ready) {
        cudaError_t e = launch_build_what(p->L, p->W64, p->What, st);
        if (e != cudaSuccess) return cuda_fail(e, "transform of W~");
        p->what_ready = true;
    }
    return MC_OK;
}

bool use_fft_full_field(const mc_lattice *p) {
    return fft_supported(p->L) && (p->path == MC_PATH_FFT || p->L >= 128);
}

// Full field of every replica into p->field: FFT for large lattices, else direct.
int full_field(mc_lattice *p, cudaStream_t st) {
    cudaError_t e;
    if (use_fft_full_field(p)) {
        int rc = ensure_fft(p, st);
        if (rc) return rc;
        TimedLaunch tl(p, MC_K_FULL_FIELD, st);
        e = launch_fft_field(p->L, p->R, p->spins, p->What, p->fft_scratch, p->field, st);
    } else {
        TimedLaunch tl(p, MC_K_FULL_FIELD, st);
        e = launch_full_field(p->L, p->R, p->W32, p->spins, p->field, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "full-field evaluation");
    return MC_OK;
}

int run_fft(mc_lattice *p, int nsweeps, int measure_every, float *trace, cudaStream_t st) {
    int rc = ensure_fft(p, st);
    if (rc) return rc;
    const int ll = p->l * p->l;
    FftStepConfig c{};
    c.t_dev = p->t_dev;
    c.L = p->L; c.l = p->l; c.R = p->R;
    c.key = key_of(p->seed);
    c.nsweeps_call = nsweeps;
    c.proposal = p->proposal;
    c.cap_c1 = (float)(1.0 - std::cos(p->cone));
    c.schedule = p->schedule;
    FftStepBuffers b{};
    b.W32 = p->W32; b.spins = p->spins; b.field = p->field; b.params = p->dparams; b.obs = p->obs;
    b.trace = trace;
    b.slots = p->packed ? p->slots_dev : nullptr;
    bool measured_last = false;
    for (int it = 0; it < nsweeps; ++it) {
        c.t = (uint32_t)(p->t + (uint64_t)it);
        c.it = it;
        for (int k = 0; k < ll; ++k) {
            cudaError_t e;
            {
                TimedLaunch tl(p, MC_K_FULL_FIELD, st);
                e = launch_fft_field(p->L, p->R, p->spins, p->What, p->fft_scratch, p->field, st);
            }
            if (e != cudaSuccess) return cuda_fail(e, "FFT field");
            c.k = k;
            {
                TimedLaunch tl(p, MC_K_WINDOW_STEPS, st);
                e = launch_fft_update(c, b, st);
            }
            if (e != cudaSuccess) return cuda_fail(e, "FFT update kernel");
        }
        // a pack measures every sweep; each slot decides from its own sweep count
        measured_last = measure_every > 0 && (b.slots || ((it + 1) % measure_every) == 0);
        if (measured_last) {
            cudaError_t e = launch_fft_field(p->L, p->R, p->spins, p->What, p->fft_scratch, p->field, st);
            if (e != cudaSuccess) return cuda_fail(e, "FFT field");
            e = launch_fft_observe(p->L, p->R, p->spins, p->field, p->dparams, p->energy, p->obs, p->theta2,
                                   b.slots, it, measure_every, hist_of(p), st);
            if (e != cudaSuccess) return cuda_fail(e, "observables");
        }
    }
    cudaError_t e = launch_add_attempted(p->obs, p->R, (long long)nsweeps * p->N(), b.slots, nsweeps, p->N(), st);
    if (e != cudaSuccess) return cuda_fail(e, "acceptance counters");
    // the FFT path does not track the energy between measurements
    p->energy_valid = p->packed || measured_last;
    return MC_OK;
}

int ensure_cluster(mc_lattice *p, cudaStream_t st) {
    const size_t K2 = (size_t)p->L / 2 + 1;
    if (!p->cl_What) CKA(cudaMalloc(&p->cl_What, sizeof(float) * 4 * K2 * p->L));
    if (!p->cl_S) {
        CKA(cudaMalloc(&p->cl_S, sizeof(float2) * (size_t)p->R * 3 * K2 * p->L));
        CKA(cudaMalloc(&p->cl_rows, sizeof(float2) * (size_t)p->R * 3 * K2 * p->L));
    }
    if (!p->cl_ready) {
        cudaError_t e = launch_cluster_what(p->L, p->W64, p->cl_What, st);
        if (e != cudaSuccess) return cuda_fail(e, "half-plane transform of W~");
        p->cl_ready = true;
    }
    return MC_OK;
}

// Cluster-resident transform path: per sweep, the 2D DFT of the spins, then one
// cluster launch for the sweep's l^2 sub-steps; the energy and observables of a
// measured sweep from a full field, as on the FFT path.
int run_cluster(mc_lattice *p, int nsweeps, int measure_every, float *trace, cudaStream_t st) {
    int rc = ensure_cluster(p, st);
    if (rc) return rc;
    ClusterSweepArgs a{};
    a.L = p->L; a.l = p->l; a.R = p->R;
    a.key = key_of(p->seed);
    a.t_dev = p->t_dev;
    a.nsweeps_call = nsweeps;
    a.proposal = p->proposal;
    a.cap_c1 = (float)(1.0 - std::cos(p->cone));
    a.schedule = p->schedule;
    a.What = p->cl_What; a.Shat = p->cl_S; a.spins = p->spins; a.W32 = p->W32;
    a.params = p->dparams; a.obs = p->obs; a.trace = trace;
    bool measured_last = false;
    for (int it = 0; it < nsweeps; ++it) {
        a.t = (uint32_t)(p->t + (uint64_t)it);
        a.it = it;
        cudaError_t e;
        {
            TimedLaunch tl(p, MC_K_FULL_FIELD, st);
            e = launch_cluster_transform(p->L, p->R, p->spins, p->cl_rows, p->cl_S, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "transform of the spins");
        {
            TimedLaunch tl(p, MC_K_SPEC_UPDATE, st);
            e = launch_cluster_sweep(a, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "cluster sweep launch");
        measured_last = measure_every > 0 && ((it + 1) % measure_every) == 0;
        if (measured_last) {
            rc = full_field(p, st);
            if (rc) return rc;
            e = launch_fft_observe(p->L, p->R, p->spins, p->field, p->dparams, p->energy, p->obs, p->theta2, nullptr,
                                   it, measure_every, hist_of(p), st);
            if (e != cudaSuccess) return cuda_fail(e, "observables");
        }
    }
    cudaError_t e = launch_add_attempted(p->obs, p->R, (long long)nsweeps * p->N(), nullptr, nsweeps, p->N(), st);
    if (e != cudaSuccess) return cuda_fail(e, "acceptance counters");
    p->energy_valid = measured_last;
    return MC_OK;
}

int ensure_spectral(mc_lattice *p, cudaStream_t st) {
    // the kernels divide (replica, K) indices below R n by n with a multiply-high
    if ((unsigned long long)p->R * p->n() * p->n() >= (1ull << 32))
        return fail(MC_ENOSYS, "spectral path needs replicas * (L/l)^4 < 2^32");
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int es = spectral_esplit(p->L, p->l, p->R, nsm);
    if (!p->specT) CKA(cudaMalloc(&p->specT, sizeof(float2) * 16 * (size_t)p->N()));
    if (!p->specS) CKA(cudaMalloc(&p->specS, sizeof(float2) * spectral_S_elems(p->L, p->R)));
    if (!p->specOff) CKA(cudaMalloc(&p->specOff, sizeof(int) * (size_t)p->R * p->l * p->l));
    if (p->spec_esplit != es) {
        cudaFree(p->specH);
        p->specH = nullptr;
        CKA(cudaMalloc(&p->specH, sizeof(float2) * spectral_part_elems(p->L, p->l, p->R, es)));
        p->spec_esplit = es;
    }
    if (!p->spec_ready) {
        cudaError_t e = launch_spec_table(p->L, p->l, p->W64, p->specT, st);
        if (e != cudaSuccess) return cuda_fail(e, "spectral W~ table");
        p->spec_ready = true;
    }
    return MC_OK;
}

// Sub-lattice spectral path: spectra of every offset from the spins, then per
// window of sub-steps the field spectra at its offsets and the update; the energy
// and observables from a full field at measured sweeps (as the FFT path).
int run_spectral(mc_lattice *p, int nsweeps, int measure_every, float *trace, cudaStream_t st) {
    int rc = ensure_spectral(p, st);
    if (rc) return rc;
    const int ll = p->l * p->l;
    SpecConfig c{};
    c.t_dev = p->t_dev;
    c.L = p->L; c.l = p->l; c.R = p->R;
    c.key = key_of(p->seed);
    c.nsweeps_call = nsweeps;
    c.proposal = p->proposal;
    c.cap_c1 = (float)(1.0 - std::cos(p->cone));
    c.schedule = p->schedule;
    c.esplit = p->spec_esplit;
    c.mC = fastdiv_magic((uint32_t)(p->L / p->l));
    c.mn = fastdiv_magic((uint32_t)p->n());
    SpecBuffers b;
    b.W32 = p->W32; b.spins = p->spins; b.params = p->dparams; b.obs = p->obs; b.trace = trace;
    b.slots = p->packed ? p->slots_dev : nullptr;
    b.T = p->specT; b.S = p->specS; b.off = p->specOff;
    c.wmax = spectral_window(p->L, p->l);
    b.Hw = p->specH;
    cudaError_t e = launch_spec_init(p->L, p->l, p->R, p->spins, p->specS, st);
    if (e != cudaSuccess) return cuda_fail(e, "spectra of the spin sub-lattices");
    // Per window of wmax sub-steps: the field spectra of its offsets from the spectra
    // at its start, then the update, which adds the window's own changes sub-step by
    // sub-step.
    bool measured_last = false;
    for (int it = 0; it < nsweeps; ++it) {
        c.t = (uint32_t)(p->t + (uint64_t)it);
        c.it = it;
        e = launch_spec_offsets(c, b, st);
        if (e != cudaSuccess) return cuda_fail(e, "sub-step offsets");
        for (int k0 = 0; k0 < ll; k0 += c.wmax) {
            c.k = k0;
            c.wlen = std::min(c.wmax, ll - k0);
            {
                TimedLaunch tl(p, MC_K_SPEC_FIELD, st);
                e = launch_spec_wfield(c, b, st);
            }
            if (e != cudaSuccess) return cuda_fail(e, "spectral field");
            {
                TimedLaunch tl(p, MC_K_SPEC_UPDATE, st);
                e = launch_spec_wupdate(c, b, st);
            }
            if (e != cudaSuccess) return cuda_fail(e, "spectral update");
        }
        measured_last = measure_every > 0 && (b.slots || ((it + 1) % measure_every) == 0);
        if (measured_last) {
            rc = full_field(p, st);
            if (rc) return rc;
            e = launch_fft_observe(p->L, p->R, p->spins, p->field, p->dparams, p->energy, p->obs, p->theta2,
                                   b.slots, it, measure_every, hist_of(p), st);
            if (e != cudaSuccess) return cuda_fail(e, "observables");
        }
    }
    e = launch_add_attempted(p->obs, p->R, (long long)nsweeps * p->N(), b.slots, nsweeps, p->N(), st);
    if (e != cudaSuccess) return cuda_fail(e, "acceptance counters");
    p->energy_valid = p->packed || measured_last;
    return MC_OK;
}

// Incremental path: launches of at most kIncrChunk sweeps, each starting from a
// freshly evaluated full field (so FP32 rank-n updates do not accumulate).
constexpr int kIncrChunk = 8;

int run_incremental(mc_lattice *p, int nsweeps, int measure_every, float *trace, cudaStream_t st) {
    IncrConfig c{};
    c.L = p->L; c.l = p->l; c.R = p->R;
    c.key = key_of(p->seed);
    c.nsweeps_call = nsweeps;
    c.measure_every = measure_every;
    c.proposal = p->proposal;
    c.cap_c1 = (float)(1.0 - std::cos(p->cone));
    c.schedule = p->schedule;
    IncrBuffers b;
    b.W32 = p->W32; b.spins = p->spins; b.field = p->field; b.params = p->dparams; b.energy = p->energy;
    b.obs = p->obs; b.theta2 = p->theta2; b.trace = trace; b.hist = hist_of(p);
    bool measured_last = false;
    for (int done = 0; done < nsweeps; done += kIncrChunk) {
        const int chunk = std::min(kIncrChunk, nsweeps - done);
        cudaError_t e;
        {
            TimedLaunch tl(p, MC_K_FULL_FIELD, st);
            e = launch_full_field(p->L, p->R, p->W32, p->spins, p->field, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "full-field kernel");
        c.t0 = (uint32_t)(p->t + (uint64_t)done);
        c.nsweeps = chunk;
        c.it0 = done;
        {
            TimedLaunch tl(p, MC_K_SWEEP_DIRECT, st);
            e = launch_sweep_incremental(c, b, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "incremental sweep kernel");
    }
    measured_last = measure_every > 0 && nsweeps % measure_every == 0;
    p->energy_valid = measured_last;
    return MC_OK;
}

int run_path(mc_lattice *p, int path, int nsweeps, int measure_every, float *trace, cudaStream_t st) {
    if (path == MC_PATH_FFT) return run_fft(p, nsweeps, measure_every, trace, st);
    if (path == MC_PATH_FFT_CLUSTER) return run_cluster(p, nsweeps, measure_every, trace, st);
    if (path == MC_PATH_SPECTRAL) return run_spectral(p, nsweeps, measure_every, trace, st);
    return run_windows(p, path, nsweeps, measure_every, trace, st);
}

// The windowed and FFT paths launch several kernels per window or sub-step.  The
// first call of a given (path, nsweeps, measure_every) runs them directly; later
// calls replay a CUDA graph of the whole call, captured on a library stream that
// is joined to the caller's stream by events.  Kernels read the sweep counter
// from t_dev, set before each call, so one graph serves every call of its shape.
int run_multi(mc_lattice *p, int path, int nsweeps, int measure_every, float *trace, cudaStream_t st) {
    if (!p->t_dev) CKA(cudaMalloc(&p->t_dev, sizeof(uint32_t)));
    cudaError_t e = launch_set_u32(p->t_dev, (uint32_t)p->t, st);
    if (e != cudaSuccess) return cuda_fail(e, "sweep counter");
    const bool graphable = !trace && !p->timing;
    const auto key = std::make_tuple(path, nsweeps, measure_every);
    // a pack repeats its quantum: capture at once; a lone handle captures a
    // shape on its second call
    if (!graphable || (p->seen[key]++ == 0 && !p->packed)) return run_path(p, path, nsweeps, measure_every, trace, st);
    if (!p->own) {
        CKA(cudaStreamCreateWithFlags(&p->own, cudaStreamNonBlocking));
        CKA(cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming));
        CKA(cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming));
    }
    auto it = p->graphs.find(key);
    if (it == p->graphs.end()) {
        // buffers and tables are made outside the capture
        if (path == MC_PATH_FFT || ((path == MC_PATH_SPECTRAL || path == MC_PATH_FFT_CLUSTER) && use_fft_full_field(p))) {
            int rc = ensure_fft(p, st);
            if (rc) return rc;
        }
        if (path == MC_PATH_FFT_CLUSTER) {
            int rc = ensure_cluster(p, st);
            if (rc) return rc;
        }
        if (path == MC_PATH_SPECTRAL) {
            int rc = ensure_spectral(p, st);
            if (rc) return rc;
        }
        cudaGraph_t g = nullptr;
        CKA(cudaStreamBeginCapture(p->own, cudaStreamCaptureModeThreadLocal));
        int rc = run_path(p, path, nsweeps, measure_every, nullptr, p->own);
        cudaError_t ec = cudaStreamEndCapture(p->own, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();  // the failed capture's error must not reach later launches
            return rc;
        }
        if (ec != cudaSuccess) return cuda_fail(ec, "graph capture");
        cudaGraphExec_t ex = nullptr;
        ec = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ec != cudaSuccess) return cuda_fail(ec, "graph instantiate");
        it = p->graphs.emplace(key, ex).first;
    }
    CKA(cudaEventRecord(p->ev_in, st));
    CKA(cudaStreamWaitEvent(p->own, p->ev_in, 0));
    CKA(cudaGraphLaunch(it->second, p->own));
    CKA(cudaEventRecord(p->ev_out, p->own));
    CKA(cudaStreamWaitEvent(st, p->ev_out, 0));
    if (path == MC_PATH_FFT || path == MC_PATH_SPECTRAL || path == MC_PATH_FFT_CLUSTER)
        p->energy_valid = p->packed || (measure_every > 0 && nsweeps % measure_every == 0);
    return MC_OK;
}

int run_sweeps(mc_lattice *p, int nsweeps, int measure_every, float *trace, cudaStream_t st) {
    if (!p->W_ready) return fail(MC_ENOTREADY, "mc_precompute_W has not been called");
    if (nsweeps < 0) return fail(MC_EINVAL, "nsweeps must be >= 0");
    if (measure_every < 0) return fail(MC_EINVAL, "measure_every must be >= 0");
    if (nsweeps == 0) return MC_OK;
    const int path0 = resolve_path(p);
    if (!p->energy_valid && path0 != MC_PATH_FFT && path0 != MC_PATH_SPECTRAL && path0 != MC_PATH_INCREMENTAL &&
        path0 != MC_PATH_FFT_CLUSTER) {
        int rc = anchor_energy(p, st);
        if (rc) return rc;
    }
    SweepConfig c;
    c.L = p->L;
    c.l = p->l;
    c.R = p->R;
    c.key = key_of(p->seed);
    c.t0 = (uint32_t)p->t;
    c.nsweeps = nsweeps;
    c.measure_every = measure_every;
    c.proposal = p->proposal;
    c.cap_c1 = (float)(1.0 - std::cos(p->cone));
    c.schedule = p->schedule;
    SweepBuffers b;
    b.W32 = p->W32;
    b.spins = p->spins;
    b.params = p->dparams;
    b.energy = p->energy;
    b.obs = p->obs;
    b.theta2 = p->theta2;
    b.trace = trace;
    b.hist = hist_of(p);
    const int path = resolve_path(p);
    if (path < 0 || !path_supported(p, path))
        return fail(MC_ENOSYS, "no field path supports L=%d l=%d (path %d)", p->L, p->l, p->path);
    if (path == MC_PATH_INCREMENTAL) {
        int rc = run_incremental(p, nsweeps, measure_every, trace, st);
        if (rc) return rc;
    } else if (path == MC_PATH_DIRECT) {
        cudaError_t e;
        {
            TimedLaunch tl(p, MC_K_SWEEP_DIRECT, st);
            e = launch_sweep_direct(c, b, p->threads_hint, st);
        }
        if (e == cudaErrorNotSupported)
            return fail(MC_ENOSYS, "no field path supports L=%d l=%d (path %d)", p->L, p->l, p->path);
        if (e != cudaSuccess) return cuda_fail(e, "sweep kernel launch");
    } else {
        int rc = run_multi(p, path, nsweeps, measure_every, trace, st);
        if (rc) return rc;
    }
    p->t += (uint64_t)nsweeps;
    p->last = st;
    return MC_OK;
}

// One grouped launch of the direct kernel over every replica (or, for a pack,
// every slot with sweeps to run) of several handles whose L / l agree: the
// descriptors go to the device through the first handle's pinned staging, and
// each CTA runs the arithmetic of its own handle's lone launch (mc_sweep, or a
// packed launch), so every replica's result is the one it has there.  For packs,
// nsweeps is each slot's own count (slots_host); `launched` = the largest.
// Launch shape of a group: the largest lone thread count and EPT of its handles and
// the shared memory of its largest lattice at that thread count.
bool group_shape(mc_lattice *const *lats, int count, int *max_nt, int *max_ept, size_t *smem) {
    *max_nt = 0;
    *max_ept = 0;
    *smem = 0;
    for (int i = 0; i < count; ++i) {
        int th = 0, ept = 0;
        if (!direct_lone_shape(lats[i]->L, lats[i]->l, lats[i]->packed ? 1 : lats[i]->R, &th, &ept)) return false;
        *max_nt = std::max(*max_nt, th);
        *max_ept = std::max(*max_ept, ept);
    }
    for (int i = 0; i < count; ++i) *smem = std::max(*smem, direct_smem_bytes(lats[i]->L, lats[i]->l, *max_nt));
    return true;
}

int run_group(mc_lattice *const *lats, int count, int nsweeps, int measure_every, cudaStream_t st, int *launched) {
    mc_lattice *h0 = lats[0];
    const int C = h0->L / h0->l;
    std::vector<SlotGeom> g;
    int max_nt = 0, max_ept = 0, mx = 0;
    size_t smem = 0;
    for (int i = 0; i < count; ++i) {
        mc_lattice *p = lats[i];
        int th = 0, ept = 0;
        if (!direct_lone_shape(p->L, p->l, p->packed ? 1 : p->R, &th, &ept))
            return fail(MC_ENOSYS, "the direct kernel does not serve L=%d l=%d", p->L, p->l);
        max_nt = std::max(max_nt, th);
        max_ept = std::max(max_ept, ept);
        const uint2 key = key_of(p->seed);
        for (int r = 0; r < p->R; ++r) {
            SlotGeom d{};
            d.L = p->L;
            d.l = p->l;
            d.nft = th - 32;
            d.nt = th;
            if (p->packed) {
                const SlotState &sl = p->slots_host[r];
                if (sl.nsweeps <= 0) continue;
                d.key_lo = sl.key_lo;
                d.key_hi = sl.key_hi;
                d.t0 = sl.t0;
                d.rid = sl.rid;
                d.nsweeps = sl.nsweeps;
                d.mphase = sl.t0;
            } else {
                d.key_lo = key.x;
                d.key_hi = key.y;
                d.t0 = (uint32_t)p->t;
                d.rid = (uint32_t)r;
                d.nsweeps = nsweeps;
                d.mphase = 0;
            }
            const size_t N = p->N();
            d.W32 = p->W32;
            d.spins = p->spins + (size_t)r * 3 * N;
            d.params = p->dparams + r;
            d.energy = p->energy + r;
            d.obs = p->obs + r;
            d.theta2 = p->theta2 + (size_t)r * N;
            mx = std::max(mx, d.nsweeps);
            g.push_back(d);
        }
    }
    *launched = mx;
    if (g.empty() || mx == 0) return MC_OK;
    group_shape(lats, count, &max_nt, &max_ept, &smem);
    const int n = (int)g.size();
    if (h0->geom_cap < n) {
        if (h0->geom_copied) CK(cudaEventSynchronize(h0->geom_copied));
        cudaFree(h0->geom_dev);
        cudaFreeHost(h0->geom_pin);
        h0->geom_dev = nullptr;
        h0->geom_pin = nullptr;
        h0->geom_cap = 0;
        CK(cudaMalloc(&h0->geom_dev, sizeof(SlotGeom) * n));
        CK(cudaMallocHost(&h0->geom_pin, sizeof(SlotGeom) * n));
        h0->geom_cap = n;
    }
    if (!h0->geom_copied) CK(cudaEventCreateWithFlags(&h0->geom_copied, cudaEventDisableTiming));
    CK(cudaEventSynchronize(h0->geom_copied));   // the previous call's staging copy is done
    std::memcpy(h0->geom_pin, g.data(), sizeof(SlotGeom) * n);
    CK(cudaMemcpyAsync(h0->geom_dev, h0->geom_pin, sizeof(SlotGeom) * n, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(h0->geom_copied, st));
    SweepConfig c{};
    c.L = h0->L;
    c.l = h0->l;
    c.nsweeps = mx;
    c.measure_every = measure_every;
    c.proposal = h0->proposal;
    c.cap_c1 = (float)(1.0 - std::cos(h0->cone));
    c.schedule = h0->schedule;
    cudaError_t e;
    {
        TimedLaunch tl(h0, MC_K_SWEEP_DIRECT, st);
        e = launch_sweep_direct_grouped(C, max_ept, max_nt, smem, c, h0->geom_dev, n, st);
    }
    if (e == cudaErrorNotSupported) return fail(MC_ENOSYS, "no direct-kernel instance covers this group");
    if (e != cudaSuccess) return cuda_fail(e, "grouped sweep launch");
    return MC_OK;
}

}  // namespace

extern "C" {

const char *mc_last_error(void) { return g_err.c_str(); }

int mc_version(void) { return kVersion; }

int mc_create_lattice(int L, int l, int replicas, uint64_t seed, mc_lattice **out) {
    g_err.clear();
    if (!out) return fail(MC_EINVAL, "out is null");
    *out = nullptr;
    if (L < 2 || L > 4096) return fail(MC_EINVAL, "L=%d outside [2, 4096]", L);
    if (l < 2 || l > L || L % l) return fail(MC_EINVAL, "l=%d must satisfy 2 <= l <= L and L %% l == 0 (L=%d)", l, L);
    if (replicas < 1) return fail(MC_EINVAL, "replicas=%d must be >= 1", replicas);
    mc_lattice *p = new mc_lattice();
    p->L = L;
    p->l = l;
    p->R = replicas;
    p->seed = seed;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaGetDevice"); }
    const size_t N = (size_t)L * L, R = replicas;
    RepParams d{};
    d.J = 1.0f; d.CD = 0.1f; d.K2 = 0.8f; d.K4 = 0.0f; d.T = 0.6f;
    p->hp.assign(R, d);
#define ALLOC(ptr, bytes)                                                            \
    do {                                                                             \
        e = cudaMalloc((void **)&(ptr), (bytes));                                    \
        if (e != cudaSuccess) {                                                      \
            free_all(p);                                                             \
            delete p;                                                                \
            cudaGetLastError();                                                      \
            return fail(MC_ENOMEM, "cudaMalloc of %zu bytes failed", (size_t)(bytes)); \
        }                                                                            \
    } while (0)
    ALLOC(p->dparams, sizeof(RepParams) * R);
    ALLOC(p->spins, sizeof(float) * 3 * N * R);
    ALLOC(p->field, sizeof(float) * 3 * N * R);
    ALLOC(p->W64, sizeof(double) * 4 * N);
    ALLOC(p->W32, sizeof(float) * 4 * N);
    ALLOC(p->energy, sizeof(double) * R);
    ALLOC(p->etmp, sizeof(double) * R);
    ALLOC(p->obs, sizeof(ObsAcc) * R);
    ALLOC(p->theta2, sizeof(double) * N * R);
#undef ALLOC
    int rc = upload_params(p);
    if (!rc) rc = clear_obs(p, nullptr);
    if (!rc) {
        e = launch_init_spins(L, replicas, key_of(seed), 1, p->spins, nullptr);
        if (e != cudaSuccess) rc = cuda_fail(e, "init kernel");
    }
    if (!rc) {
        e = cudaMemset(p->energy, 0, sizeof(double) * R);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemset");
    }
    if (!rc) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = cuda_fail(e, "create: synchronize");
    }
    if (rc) {
        free_all(p);
        delete p;
        return rc;
    }
    *out = p;
    return MC_OK;
}

int mc_destroy(mc_lattice *p) {
    if (!p) return MC_OK;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    clear_timing(p);
    free_all(p);
    delete p;
    return MC_OK;
}

int mc_set_params(mc_lattice *p, int replica, double J, double C_D, double K2, double K4, double T) {
    int rc = check(p);
    if (rc) return rc;
    if (replica < -1 || replica >= p->R) return fail(MC_EINVAL, "replica %d out of range", replica);
    if (!(T > 0.0) || !std::isfinite(T)) return fail(MC_EINVAL, "T must be > 0 and finite");
    if (!std::isfinite(J) || !std::isfinite(C_D) || !std::isfinite(K2) || !std::isfinite(K4))
        return fail(MC_EINVAL, "couplings must be finite");
    for (int r = 0; r < p->R; ++r) {
        if (replica >= 0 && r != replica) continue;
        RepParams &q = p->hp[r];
        q.J = (float)J; q.CD = (float)C_D; q.K2 = (float)K2; q.K4 = (float)K4; q.T = (float)T;
    }
    CK(cudaDeviceSynchronize());
    rc = upload_params(p);
    p->energy_valid = false;
    return rc;
}

int mc_set_proposal(mc_lattice *p, int kind, double cone) {
    if (p) drop_graphs(p);
    int rc = check(p);
    if (rc) return rc;
    if (kind < 0 || kind > 2) return fail(MC_EINVAL, "proposal kind must be 0, 1 or 2");
    if (kind == 0 && !(cone > 0.0 && cone <= M_PI)) return fail(MC_EINVAL, "cone must be in (0, pi]");
    p->proposal = kind;
    if (kind == 0) p->cone = cone;
    return MC_OK;
}

int mc_set_schedule(mc_lattice *p, int kind) {
    if (p) drop_graphs(p);
    int rc = check(p);
    if (rc) return rc;
    if (kind != 0 && kind != 1) return fail(MC_EINVAL, "schedule kind must be 0 or 1");
    p->schedule = kind;
    return MC_OK;
}

int mc_set_field_path(mc_lattice *p, int path) {
    if (p) drop_graphs(p);
    int rc = check(p);
    if (rc) return rc;
    if (path < MC_PATH_AUTO || path > MC_PATH_FFT_CLUSTER) return fail(MC_EINVAL, "unknown field path %d", path);
    if (path != MC_PATH_AUTO && !path_supported(p, path))
        return fail(MC_ENOSYS, "field path %d does not support L=%d l=%d", path, p->L, p->l);
    p->path = path;
    return MC_OK;
}

int mc_set_window(mc_lattice *p, int B) {
    if (p) drop_graphs(p);
    int rc = check(p);
    if (rc) return rc;
    if (B < 0 || (B > 0 && (p->l * p->l) % B)) return fail(MC_EINVAL, "window %d must divide l^2 = %d", B, p->l * p->l);
    if (B > 0 && !window_supported(p->L, p->l, B)) return fail(MC_EINVAL, "window %d too large for L=%d", B, p->L);
    p->window_B = B;
    return MC_OK;
}

int mc_set_tuning(mc_lattice *p, const mc_tuning *t) {
    int rc = check(p);
    if (rc) return rc;
    if (!t) return fail(MC_EINVAL, "null tuning");
    if (t->tc_kblocks < 0 || t->tc_kblocks > 4096) return fail(MC_EINVAL, "tc_kblocks must be in [0, 4096]");
    if (t->tc_ntile != 0 && (t->tc_ntile < 16 || t->tc_ntile > 256 || t->tc_ntile % 16))
        return fail(MC_EINVAL, "tc_ntile must be 0 or a multiple of 16 in [16, 256]");
    if (t->steps_layout < 0 || t->steps_layout > 2) return fail(MC_EINVAL, "steps_layout must be 0, 1 or 2");
    rc = mc_set_window(p, t->window);
    if (rc) return rc;
    drop_graphs(p);
    p->tc_kblocks = t->tc_kblocks;
    p->tc_ntile = t->tc_ntile;
    p->steps_layout = t->steps_layout;
    return MC_OK;
}

int mc_get_tuning(mc_lattice *p, mc_tuning *out) {
    if (!p || !out) return fail(MC_EINVAL, "null argument");
    out->window = p->window_B;
    out->tc_kblocks = p->tc_kblocks;
    out->tc_ntile = p->tc_ntile;
    out->steps_layout = p->steps_layout;
    return MC_OK;
}

int mc_init_spins(mc_lattice *p, int mode, const float *user) {
    int rc = check(p);
    if (rc) return rc;
    if (mode < 0 || mode > 3) return fail(MC_EINVAL, "init mode must be 0, 1, 2 or 3");
    CK(cudaDeviceSynchronize());
    if (mode == 2) {
        if (!user) return fail(MC_EINVAL, "mode 2 needs a host array");
        CK(cudaMemcpy(p->spins, user, sizeof(float) * p->spin_floats(), cudaMemcpyHostToDevice));
    } else {
        cudaError_t e = launch_init_spins(p->L, p->R, key_of(p->seed), mode, p->spins, nullptr);
        if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    }
    rc = clear_obs(p, nullptr);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    p->t = 0;
    p->energy_valid = false;
    return MC_OK;
}

int mc_precompute_W(mc_lattice *p, int A, int tail) {
    if (p) drop_graphs(p);
    int rc = check(p);
    if (rc) return rc;
    if (A < 0 || A > 4096) return fail(MC_EINVAL, "image_cutoff %d outside [0, 4096]", A);
    cudaError_t e = launch_wtilde(p->L, A, tail ? 1 : 0, p->W64, p->W32, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "W~ kernel");
    if (!p->wq) CK(cudaMalloc(&p->wq, sizeof(float4) * wq_table_elems(p->L)));
    e = launch_build_wq(p->L, p->W32, p->wq, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "W~ quarter table");
    CK(cudaDeviceSynchronize());
    p->A = A;
    p->tail = tail ? 1 : 0;
    p->W_ready = true;
    p->wsh_ready = false;
    p->what_ready = false;
    p->cl_ready = false;
    p->spec_ready = false;
    p->energy_valid = false;
    return MC_OK;
}

int mc_precompute_W_ewald(mc_lattice *p, double eta) {
    if (p) drop_graphs(p);
    int rc = check(p);
    if (rc) return rc;
    if (!(eta > 0.0)) eta = p->L / 4.0;
    double *W6 = nullptr;
    CK(cudaMalloc(&W6, sizeof(double) * 6 * (size_t)p->N()));
    cudaError_t e = launch_wtilde_ewald(p->L, 0.0, eta, W6, nullptr);
    if (e == cudaSuccess) e = launch_take_plane(p->L, W6, p->W64, p->W32, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(W6);
    if (e != cudaSuccess) return cuda_fail(e, "Ewald W~ kernel");
    if (!p->wq) CK(cudaMalloc(&p->wq, sizeof(float4) * wq_table_elems(p->L)));
    e = launch_build_wq(p->L, p->W32, p->wq, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "W~ quarter table");
    CK(cudaDeviceSynchronize());
    p->A = -1;
    p->tail = 0;
    p->W_ready = true;
    p->wsh_ready = false;
    p->what_ready = false;
    p->cl_ready = false;
    p->spec_ready = false;
    p->energy_valid = false;
    return MC_OK;
}

int mc_wtilde_ewald(int L, double z, double eta, double *dst) {
    g_err.clear();
    if (!dst) return fail(MC_EINVAL, "dst is null");
    if (L < 2 || L > 4096) return fail(MC_EINVAL, "L=%d outside [2, 4096]", L);
    if (!(std::fabs(z) <= (double)L)) return fail(MC_EINVAL, "|z| must be <= L");
    if (!(eta > 0.0)) eta = L / 4.0;
    const size_t n = (size_t)6 * L * L;
    double *W6 = nullptr;
    CK(cudaMalloc(&W6, sizeof(double) * n));
    cudaError_t e = launch_wtilde_ewald(L, z, eta, W6, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(dst, W6, sizeof(double) * n, cudaMemcpyDeviceToHost);
    cudaFree(W6);
    if (e != cudaSuccess) return cuda_fail(e, "Ewald W~ kernel");
    return MC_OK;
}

int mc_sweep(mc_lattice *p, int nsweeps, int measure_every, void *stream) {
    int rc = check(p);
    if (rc) return rc;
    return run_sweeps(p, nsweeps, measure_every, nullptr, (cudaStream_t)stream);
}

int mc_sweep_group(mc_lattice *const *lats, int count, int nsweeps, int measure_every, void *stream) {
    if (!lats || count < 1) return fail(MC_EINVAL, "mc_sweep_group needs at least one handle");
    if (nsweeps < 0 || measure_every < 0) return fail(MC_EINVAL, "nsweeps and measure_every must be >= 0");
    mc_lattice *h0 = lats[0];
    int rc = check(h0);
    if (rc) return rc;
    for (int i = 0; i < count; ++i) {
        mc_lattice *p = lats[i];
        if (!p) return fail(MC_EINVAL, "handle %d is null", i);
        for (int j = 0; j < i; ++j)
            if (lats[j] == p) return fail(MC_EINVAL, "handle %d appears twice", i);
        if (p->device != h0->device) return fail(MC_EINVAL, "handles of one group must be on one device");
        if (p->packed) return fail(MC_EINVAL, "handle %d is a serving pack", i);
        if (!p->W_ready) return fail(MC_ENOTREADY, "handle %d: mc_precompute_W has not been called", i);
        if (resolve_path(p) != MC_PATH_DIRECT)
            return fail(MC_EINVAL, "handle %d does not run the direct path (set MC_PATH_DIRECT)", i);
        if (p->L / p->l != h0->L / h0->l)
            return fail(MC_EINVAL, "handles of one group need the same L / l (%d vs %d)", p->L / p->l, h0->L / h0->l);
        if (p->proposal != h0->proposal || p->cone != h0->cone || p->schedule != h0->schedule)
            return fail(MC_EINVAL, "handles of one group need the same proposal, cone and schedule");
        if (p->hist) return fail(MC_EINVAL, "handle %d keeps an energy histogram (not kept in grouped launches)", i);
    }
    if (nsweeps == 0) return MC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < count; ++i)
        if (!lats[i]->energy_valid) {
            rc = anchor_energy(lats[i], st);
            if (rc) return rc;
        }
    int launched = 0;
    rc = run_group(lats, count, nsweeps, measure_every, st, &launched);
    if (rc) return rc;
    for (int i = 0; i < count; ++i) {
        lats[i]->t += (uint64_t)nsweeps;
        lats[i]->last = st;
    }
    return MC_OK;
}

int mc_sweep_trace(mc_lattice *p, int nsweeps, float *trace, size_t trace_floats, void *stream) {
    int rc = check(p);
    if (rc) return rc;
    if (!trace) return fail(MC_EINVAL, "trace buffer is null");
    const size_t need = (size_t)p->R * (size_t)nsweeps * p->N() * MC_TRACE_W;
    if (trace_floats < need) return fail(MC_EINVAL, "trace buffer holds %zu floats, needs %zu", trace_floats, need);
    return run_sweeps(p, nsweeps, 0, trace, (cudaStream_t)stream);
}

// Statistics of replicas [first, first + count) into out[]: eta reduced on the
// device, then one copy each of the accumulators, the energies and eta, on the
// lattice's last stream.
int obs_fill(mc_lattice *p, int first, int count, mc_obs *out) {
    CK(cudaStreamSynchronize(p->last));
    int rc = check_device_flag(p);
    if (rc) return rc;
    if (!p->eta_dev) CKA(cudaMalloc(&p->eta_dev, sizeof(double) * p->R));
    const int N = p->N();
    cudaError_t e = launch_eta(N, count, p->theta2 + (size_t)first * N, p->obs + first, p->eta_dev + first, p->last);
    if (e != cudaSuccess) return cuda_fail(e, "eta reduction");
    // the copies land in pinned staging (direct DMA, no per-call allocation); if pinned
    // memory cannot be had, in pageable vectors
    if (count > p->obs_pin_cap) {
        if (p->obs_pin) cudaFreeHost(p->obs_pin);
        p->obs_pin = nullptr;
        p->obs_pin_cap = 0;
        if (cudaMallocHost((void **)&p->obs_pin, (sizeof(ObsAcc) + 2 * sizeof(double)) * (size_t)count) == cudaSuccess)
            p->obs_pin_cap = count;
        else
            cudaGetLastError();
    }
    std::vector<ObsAcc> Av;
    std::vector<double> Ev, etav;
    const ObsAcc *A;
    const double *E, *eta;
    if (p->obs_pin) {
        A = reinterpret_cast<const ObsAcc *>(p->obs_pin);
        E = reinterpret_cast<const double *>(p->obs_pin + sizeof(ObsAcc) * (size_t)p->obs_pin_cap);
        eta = E + p->obs_pin_cap;
    } else {
        Av.resize((size_t)count);
        Ev.resize((size_t)count);
        etav.resize((size_t)count);
        A = Av.data(); E = Ev.data(); eta = etav.data();
    }
    CK(cudaMemcpyAsync((void *)A, p->obs + first, sizeof(ObsAcc) * count, cudaMemcpyDeviceToHost, p->last));
    CK(cudaMemcpyAsync((void *)E, p->energy + first, sizeof(double) * count, cudaMemcpyDeviceToHost, p->last));
    CK(cudaMemcpyAsync((void *)eta, p->eta_dev + first, sizeof(double) * count, cudaMemcpyDeviceToHost, p->last));
    CK(cudaStreamSynchronize(p->last));
    for (int i = 0; i < count; ++i) {
        const ObsAcc &a = A[i];
        mc_obs *o = out + i;
        std::memset(o, 0, sizeof(*o));
        const long long n = a.bcnt[0];
        o->samples = n;
        o->accepted = a.accepted;
        o->attempted = a.attempted;
        o->energy = p->energy_valid ? E[i] / N : NAN;
        for (int k = 0; k < MC_NOBS; ++k) {
            if (n < 1) { o->mean[k] = NAN; continue; }
            const double m = a.bsum[k][0] / n;
            const double v = std::fmax(0.0, a.bsq[k][0] / n - m * m);
            o->mean[k] = m;
            o->var[k] = v;
            o->err_naive[k] = n > 1 ? std::sqrt(v / (n - 1)) : NAN;
            double best = o->err_naive[k];
            for (int lv = 1; lv < kNB; ++lv) {
                const long long nb = a.bcnt[lv];
                if (nb < 32) break;
                const double mk = a.bsum[k][lv] / nb;
                const double vk = std::fmax(0.0, a.bsq[k][lv] / nb - mk * mk);
                const double ek = std::sqrt(vk / (nb - 1));
                if (ek > best) best = ek;
            }
            o->err[k] = best;
            o->tau_int[k] = (o->err_naive[k] > 0) ? 0.5 * (best / o->err_naive[k]) * (best / o->err_naive[k]) : NAN;
        }
        o->eta = eta[i];
    }
    return MC_OK;
}

int mc_observables(mc_lattice *p, int replica, mc_obs *out) {
    int rc = check(p);
    if (rc) return rc;
    if (!out) return fail(MC_EINVAL, "out is null");
    if (replica < 0 || replica >= p->R) return fail(MC_EINVAL, "replica %d out of range", replica);
    return obs_fill(p, replica, 1, out);
}

int mc_observables_batch(mc_lattice *p, int first, int count, mc_obs *out) {
    int rc = check(p);
    if (rc) return rc;
    if (!out) return fail(MC_EINVAL, "out is null");
    if (first < 0 || count < 0 || first + count > p->R)
        return fail(MC_EINVAL, "replicas [%d, %d) outside [0, %d)", first, first + count, p->R);
    if (count == 0) return MC_OK;
    return obs_fill(p, first, count, out);
}

int mc_set_histogram(mc_lattice *p, double lo, double hi, int nbins) {
    if (p) drop_graphs(p);
    int rc = check(p);
    if (rc) return rc;
    if (nbins < 0 || nbins > (1 << 20)) return fail(MC_EINVAL, "nbins %d outside [0, 2^20]", nbins);
    if (nbins > 0 && !(hi > lo)) return fail(MC_EINVAL, "histogram range needs hi > lo");
    CK(cudaDeviceSynchronize());
    cudaFree(p->hist);
    p->hist = nullptr;
    p->hist_bins = 0;
    if (nbins == 0) return MC_OK;
    CK(cudaMalloc(&p->hist, sizeof(unsigned long long) * p->R * nbins));
    CK(cudaMemset(p->hist, 0, sizeof(unsigned long long) * p->R * nbins));
    p->hist_bins = nbins;
    p->hist_lo = lo;
    p->hist_scale = (double)nbins / (hi - lo);
    return MC_OK;
}

int mc_get_histogram(mc_lattice *p, int replica, int64_t *counts) {
    int rc = check(p);
    if (rc) return rc;
    if (!counts) return fail(MC_EINVAL, "counts is null");
    if (!p->hist) return fail(MC_ENOTREADY, "no histogram set (mc_set_histogram)");
    if (replica < 0 || replica >= p->R) return fail(MC_EINVAL, "replica %d out of range", replica);
    CK(cudaStreamSynchronize(p->last));
    CK(cudaMemcpy(counts, p->hist + (size_t)replica * p->hist_bins, sizeof(int64_t) * p->hist_bins,
                  cudaMemcpyDeviceToHost));
    return MC_OK;
}

int mc_reset_observables(mc_lattice *p) {
    int rc = check(p);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    rc = clear_obs(p, nullptr);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    return MC_OK;
}

int mc_get_spins(mc_lattice *p, float *dst, int on_device, void *stream) {
    int rc = check(p);
    if (rc) return rc;
    if (!dst) return fail(MC_EINVAL, "dst is null");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(dst, p->spins, sizeof(float) * p->spin_floats(),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return check_device_flag(p);
}

int mc_get_field(mc_lattice *p, float *dst, int on_device, void *stream) {
    int rc = check(p);
    if (rc) return rc;
    if (!dst) return fail(MC_EINVAL, "dst is null");
    if (!p->W_ready) return fail(MC_ENOTREADY, "mc_precompute_W has not been called");
    cudaStream_t st = (cudaStream_t)stream;
    rc = full_field(p, st);
    if (rc) return rc;
    CK(cudaMemcpyAsync(dst, p->field, sizeof(float) * p->spin_floats(),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return MC_OK;
}

int mc_get_W(mc_lattice *p, double *dst) {
    int rc = check(p);
    if (rc) return rc;
    if (!dst) return fail(MC_EINVAL, "dst is null");
    if (!p->W_ready) return fail(MC_ENOTREADY, "mc_precompute_W has not been called");
    CK(cudaMemcpy(dst, p->W64, sizeof(double) * 4 * p->N(), cudaMemcpyDeviceToHost));
    return MC_OK;
}

int mc_energy(mc_lattice *p, double *dst, void *stream) {
    int rc = check(p);
    if (rc) return rc;
    if (!dst) return fail(MC_EINVAL, "dst is null");
    if (!p->W_ready) return fail(MC_ENOTREADY, "mc_precompute_W has not been called");
    cudaStream_t st = (cudaStream_t)stream;
    rc = full_field(p, st);
    if (rc) return rc;
    cudaError_t e = launch_energy(p->L, p->R, p->spins, p->field, p->dparams, p->etmp, st);
    if (e != cudaSuccess) return cuda_fail(e, "energy kernel");
    CK(cudaMemcpyAsync(dst, p->etmp, sizeof(double) * p->R, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return MC_OK;
}

int mc_set_timing(mc_lattice *p, int enable) {
    int rc = check(p);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    clear_timing(p);
    p->timing = enable != 0;
    if (p->timing) {
        if (!p->wcyc) CK(cudaMalloc(&p->wcyc, 4 * sizeof(unsigned long long)));
        CK(cudaMemset(p->wcyc, 0, 4 * sizeof(unsigned long long)));
    }
    return MC_OK;
}

int mc_get_window_cycles(mc_lattice *p, double *out) {
    int rc = check(p);
    if (rc) return rc;
    if (!out) return fail(MC_EINVAL, "out is null");
    unsigned long long c[4] = {0, 0, 0, 0};
    if (p->wcyc) {
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(c, p->wcyc, sizeof c, cudaMemcpyDeviceToHost));
    }
    // c[3] counts blocks over CTAs and launches; CTA-launches = blocks / blocks per launch
    const int B = window_of(p, resolve_path(p) == MC_PATH_TENSOR);
    const double nblk = (p->n() <= 16 && B > 0) ? (double)B / (16.0 / p->n()) : 0.0;   // blocks per launch
    const double ctal = (c[3] && nblk > 0) ? (double)c[3] / nblk : 0.0;                  // CTA-launches
    out[0] = c[3] ? (double)c[0] / (double)c[3] : 0.0;
    out[1] = ctal > 0 ? (double)c[1] / ctal : 0.0;
    out[2] = ctal > 0 ? (double)c[2] / ctal : 0.0;
    out[3] = nblk;
    return MC_OK;
}

int mc_get_timing(mc_lattice *p, mc_timing *out) {
    int rc = check(p);
    if (rc) return rc;
    if (!out) return fail(MC_EINVAL, "out is null");
    CK(cudaDeviceSynchronize());
    std::memset(out, 0, sizeof *out);
    for (int k = 0; k < MC_NKCLASS; ++k) {
        for (auto &e : p->tev[k]) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e.first, e.second));
            out->ms[k] += ms;
            out->launches[k] += 1;
        }
    }
    return MC_OK;
}

int mc_choose_spacing(int L, double C_D, double T_min, double max_error, int *l_out) {
    if (!l_out || L < 2 || !(T_min > 0.0) || !(max_error > 0.0)) return fail(MC_EINVAL, "bad arguments");
    constexpr double kLatticeSum = 9.033621683;   // sum over Z^2 \ 0 of |v|^-3 = 4 zeta(3/2) beta(3/2)
    for (int l = 2; l <= L; ++l) {
        if (L % l) continue;
        const double eps = 2.0 * std::fabs(C_D) * kLatticeSum / ((double)l * l * l);
        if (eps / T_min <= max_error) {
            *l_out = l;
            return MC_OK;
        }
    }
    *l_out = L;
    return MC_OK;
}

int mc_autotune(mc_lattice *p, int nsweeps_trial, void *stream, int *path_out, int *window_out) {
    int rc = check(p);
    if (rc) return rc;
    if (nsweeps_trial < 1) return fail(MC_EINVAL, "nsweeps_trial must be >= 1");
    if (!p->W_ready) return fail(MC_ENOTREADY, "mc_precompute_W has not been called");
    cudaStream_t st = (cudaStream_t)stream;
    size_t len = 0;
    rc = mc_checkpoint(p, nullptr, &len);
    if (rc) return rc;
    std::vector<char> saved(len);
    rc = mc_checkpoint(p, saved.data(), &len);
    if (rc) return rc;
    const int old_path = p->path, old_B = p->window_B;
    struct Cand { int path, B; };
    std::vector<Cand> cands;
    if (path_supported(p, MC_PATH_DIRECT)) cands.push_back({MC_PATH_DIRECT, 0});
    for (int B : {32, 64, 128}) {
        p->window_B = B;
        if ((p->l * p->l) % B == 0 && path_supported(p, MC_PATH_TENSOR)) cands.push_back({MC_PATH_TENSOR, B});
    }
    p->window_B = old_B;
    if (path_supported(p, MC_PATH_FFT)) cands.push_back({MC_PATH_FFT, 0});
    if (path_supported(p, MC_PATH_SPECTRAL)) cands.push_back({MC_PATH_SPECTRAL, 0});
    if (path_supported(p, MC_PATH_INCREMENTAL)) cands.push_back({MC_PATH_INCREMENTAL, 0});
    if (path_supported(p, MC_PATH_FFT_CLUSTER)) cands.push_back({MC_PATH_FFT_CLUSTER, 0});
    if (cands.empty()) return fail(MC_ENOSYS, "no field path supports L=%d l=%d", p->L, p->l);
    // the timing events are destroyed on every return below, early ones included
    struct EventPair {
        cudaEvent_t a = nullptr, b = nullptr;
        ~EventPair() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } events;
    CK(cudaEventCreate(&events.a));
    CK(cudaEventCreate(&events.b));
    cudaEvent_t a = events.a, b = events.b;
    float best = 1e30f;
    Cand win = cands[0];
    for (const Cand &c : cands) {
        drop_graphs(p);
        p->path = c.path;
        p->window_B = c.B;
        rc = run_sweeps(p, 1, 0, nullptr, st);                 // warm-up (allocations, attributes)
        if (!rc) {
            CK(cudaEventRecord(a, st));
            rc = run_sweeps(p, nsweeps_trial, 0, nullptr, st);
            CK(cudaEventRecord(b, st));
        }
        CK(cudaStreamSynchronize(st));
        float ms = 0.f;
        if (!rc) CK(cudaEventElapsedTime(&ms, a, b));
        if (!rc && ms < best) {
            best = ms;
            win = c;
        }
        int r2 = mc_restore(p, saved.data(), len);
        if (r2) return r2;
    }
    drop_graphs(p);
    (void)old_path;
    p->path = win.path;
    p->window_B = win.B;
    if (win.path == MC_PATH_TENSOR) {
        // launch shapes of the tensor path, one field at a time (coordinate search),
        // each candidate timed as above; a candidate that fails is skipped
        auto trial = [&](float *ms) -> int {
            drop_graphs(p);
            int r = run_sweeps(p, 1, 0, nullptr, st);
            if (!r) {
                CK(cudaEventRecord(a, st));
                r = run_sweeps(p, nsweeps_trial, 0, nullptr, st);
                CK(cudaEventRecord(b, st));
            }
            CK(cudaStreamSynchronize(st));
            if (!r) CK(cudaEventElapsedTime(ms, a, b));
            int r2 = mc_restore(p, saved.data(), len);
            if (r2) return r2;
            return r;
        };
        int *fields[3] = {&p->tc_kblocks, &p->tc_ntile, &p->steps_layout};
        const std::vector<int> choices[3] = {{0, 2, 4, 6, 8, 12}, {0, 128}, {0, 1, 2}};
        for (int f = 0; f < 3; ++f) {
            int keep = *fields[f];
            float bf = 1e30f;
            for (int v : choices[f]) {
                *fields[f] = v;
                float ms = 0.f;
                const int r = trial(&ms);
                if (r == MC_ETIMEOUT || r == MC_ECUDA) return r;
                if (!r && ms < bf) {
                    bf = ms;
                    keep = v;
                }
            }
            *fields[f] = keep;
        }
        drop_graphs(p);
    }
    if (path_out) *path_out = win.path;
    if (window_out) *window_out = win.B;
    return MC_OK;
}

int mc_get_sweep_counter(mc_lattice *p, uint64_t *out) {
    if (!p || !out) return fail(MC_EINVAL, "null argument");
    *out = p->t;
    return MC_OK;
}

namespace {
struct CkptHeader {
    uint32_t magic;
    int32_t version, L, l, R, proposal, schedule, A, tail, W_ready, energy_valid, pad;
    uint64_t seed, t;
    double cone;
};
}  // namespace

int mc_checkpoint(mc_lattice *p, void *buf, size_t *len) {
    int rc = check(p);
    if (rc) return rc;
    if (!len) return fail(MC_EINVAL, "len is null");
    const size_t N = p->N(), R = p->R;
    const size_t need = sizeof(CkptHeader) + sizeof(RepParams) * R + sizeof(float) * 3 * N * R +
                        sizeof(double) * R + sizeof(ObsAcc) * R + sizeof(double) * N * R;
    if (!buf) { *len = need; return MC_OK; }
    if (*len < need) return fail(MC_EINVAL, "checkpoint buffer too small (%zu < %zu)", *len, need);
    CK(cudaDeviceSynchronize());
    char *o = (char *)buf;
    CkptHeader h{};
    h.magic = kMagic; h.version = kVersion; h.L = p->L; h.l = p->l; h.R = p->R;
    h.proposal = p->proposal; h.schedule = p->schedule; h.A = p->A; h.tail = p->tail;
    h.W_ready = p->W_ready; h.energy_valid = p->energy_valid; h.seed = p->seed; h.t = p->t; h.cone = p->cone;
    std::memcpy(o, &h, sizeof h); o += sizeof h;
    std::memcpy(o, p->hp.data(), sizeof(RepParams) * R); o += sizeof(RepParams) * R;
    CK(cudaMemcpy(o, p->spins, sizeof(float) * 3 * N * R, cudaMemcpyDeviceToHost)); o += sizeof(float) * 3 * N * R;
    CK(cudaMemcpy(o, p->energy, sizeof(double) * R, cudaMemcpyDeviceToHost)); o += sizeof(double) * R;
    CK(cudaMemcpy(o, p->obs, sizeof(ObsAcc) * R, cudaMemcpyDeviceToHost)); o += sizeof(ObsAcc) * R;
    CK(cudaMemcpy(o, p->theta2, sizeof(double) * N * R, cudaMemcpyDeviceToHost));
    *len = need;
    return MC_OK;
}

int mc_restore(mc_lattice *p, const void *buf, size_t len) {
    int rc = check(p);
    if (rc) return rc;
    if (!buf || len < sizeof(CkptHeader)) return fail(MC_EINVAL, "checkpoint buffer too small");
    CkptHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (h.magic != kMagic || h.version != kVersion) return fail(MC_EINVAL, "not a dipmc checkpoint");
    if (h.L != p->L || h.l != p->l || h.R != p->R)
        return fail(MC_EINVAL, "checkpoint is for L=%d l=%d R=%d, handle has L=%d l=%d R=%d", h.L, h.l, h.R, p->L, p->l, p->R);
    const size_t N = p->N(), R = p->R;
    const size_t need = sizeof(CkptHeader) + sizeof(RepParams) * R + sizeof(float) * 3 * N * R +
                        sizeof(double) * R + sizeof(ObsAcc) * R + sizeof(double) * N * R;
    if (len < need) return fail(MC_EINVAL, "checkpoint truncated (%zu < %zu)", len, need);
    if (h.proposal < 0 || h.proposal > 2 || (h.schedule != 0 && h.schedule != 1) || !(h.cone > 0.0 && h.cone <= M_PI))
        return fail(MC_EINVAL, "checkpoint holds an invalid proposal kind, schedule or cone");
    if (h.W_ready && (!p->W_ready || h.A != p->A || h.tail != p->tail))
        return fail(MC_ENOTREADY, "call mc_precompute_W(%d, %d) on this handle before mc_restore", h.A, h.tail);
    CK(cudaDeviceSynchronize());
    // the captured launch graphs hold the seed's key, the proposal kind, the cone and the
    // schedule as kernel arguments; the checkpoint may carry other ones
    drop_graphs(p);
    const char *o = (const char *)buf + sizeof h;
    std::memcpy(p->hp.data(), o, sizeof(RepParams) * R); o += sizeof(RepParams) * R;
    rc = upload_params(p);
    if (rc) return rc;
    CK(cudaMemcpy(p->spins, o, sizeof(float) * 3 * N * R, cudaMemcpyHostToDevice)); o += sizeof(float) * 3 * N * R;
    CK(cudaMemcpy(p->energy, o, sizeof(double) * R, cudaMemcpyHostToDevice)); o += sizeof(double) * R;
    CK(cudaMemcpy(p->obs, o, sizeof(ObsAcc) * R, cudaMemcpyHostToDevice)); o += sizeof(ObsAcc) * R;
    CK(cudaMemcpy(p->theta2, o, sizeof(double) * N * R, cudaMemcpyHostToDevice));
    p->seed = h.seed;
    p->t = h.t;
    p->proposal = h.proposal;
    p->schedule = h.schedule;
    p->cone = h.cone;
    p->energy_valid = h.energy_valid != 0;
    return MC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Internal entry points of the serving layer (server.cu).  None is exported.
// ---------------------------------------------------------------------------
namespace dipmc {

// W~ (FP64, device) computed once for (L, cutoff) and copied into the handle with
// its derived tables; equivalent to mc_precompute_W(p, A, tail).
int lattice_copy_W(mc_lattice *p, const double *W64_dev, int A, int tail) {
    int rc = check(p);
    if (rc) return rc;
    drop_graphs(p);
    CK(cudaMemcpy(p->W64, W64_dev, sizeof(double) * 4 * (size_t)p->N(), cudaMemcpyDeviceToDevice));
    cudaError_t e = launch_cast_W(p->L, p->W64, p->W32, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "W~ cast");
    if (!p->wq) CK(cudaMalloc(&p->wq, sizeof(float4) * wq_table_elems(p->L)));
    e = launch_build_wq(p->L, p->W32, p->wq, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "W~ quarter table");
    CK(cudaDeviceSynchronize());
    p->A = A;
    p->tail = tail ? 1 : 0;
    p->W_ready = true;
    p->wsh_ready = false;
    p->what_ready = false;
    p->cl_ready = false;
    p->spec_ready = false;
    p->energy_valid = false;
    return MC_OK;
}

// Device bytes of a handle on the path its (L, l) resolves to automatically.
size_t lattice_footprint(int L, int l, int R) {
    const size_t N = (size_t)L * L, hq = (size_t)(L / 2 + 1);
    size_t b = sizeof(RepParams) * R + sizeof(float) * 3 * N * R * 2 + sizeof(double) * 4 * N +
               sizeof(float) * 4 * N + sizeof(double) * 2 * R + sizeof(ObsAcc) * R + sizeof(double) * N * R +
               sizeof(float4) * hq * hq + sizeof(SlotState) * R;
    if (fft_supported(L) && (!direct_supported(L, l) || L >= 64))   // FFT path or FFT energy anchor
        b += sizeof(float) * 4 * N + fft_scratch_bytes(L, R) + sizeof(double2) * 4 * N;
    if ((!direct_supported(L, l) || L >= 128) && spectral_supported(L, l)) {
        const int es = spectral_esplit(L, l, R, 148);
        b += sizeof(float2) * (16 * N + spectral_S_elems(L, R) + spectral_part_elems(L, l, R, std::max(es, 16)));
    }
    return b + 4096;
}

int lattice_resolved_path(mc_lattice *p) { return resolve_path(p); }

// Turn a fresh handle (direct path) into a pack of independent replica slots.
int pack_enable(mc_lattice *p, int path) {
    int rc = check(p);
    if (rc) return rc;
    const bool ok = path == MC_PATH_DIRECT     ? direct_supported(p->L, p->l)
                    : path == MC_PATH_FFT      ? fft_supported(p->L)
                    : path == MC_PATH_SPECTRAL ? spectral_supported(p->L, p->l)
                                               : false;
    if (!ok) return fail(MC_ENOSYS, "packed launches need the direct, FFT or spectral path");
    CK(cudaMalloc(&p->slots_dev, sizeof(SlotState) * p->R));
    CK(cudaMallocHost(&p->slots_pin, sizeof(SlotState) * p->R));
    CK(cudaMallocHost(&p->params_pin, sizeof(RepParams) * p->R));
    CK(cudaEventCreateWithFlags(&p->slots_copied, cudaEventDisableTiming));
    p->slots_host.assign(p->R, SlotState{});
    p->packed = true;
    p->path = path;
    p->energy_valid = true;  // direct: anchored when a slot is filled; FFT: set at measurements
    return MC_OK;
}

// Fill slots [slot, slot + count) with one request: its couplings, its seed and
// spins initialised exactly as mc_init_spins does for a lone lattice of `count`
// replicas, cleared accumulators and an anchored energy.  Stream-ordered on st.
int pack_fill(mc_lattice *p, int slot, int count, uint64_t seed, const RepParams &rp, int init_mode,
              cudaStream_t st) {
    if (!p->packed || slot < 0 || count < 1 || slot + count > p->R) return fail(MC_EINVAL, "bad slot range");
    const uint2 key = key_of(seed);
    for (int i = 0; i < count; ++i) {
        p->params_pin[slot + i] = rp;
        p->hp[slot + i] = rp;
        SlotState s{};
        s.key_lo = key.x;
        s.key_hi = key.y;
        s.rid = (uint32_t)i;
        p->slots_host[slot + i] = s;
    }
    const size_t N = p->N(), off = (size_t)slot * 3 * N;
    CK(cudaMemcpyAsync(p->dparams + slot, p->params_pin + slot, sizeof(RepParams) * count, cudaMemcpyHostToDevice, st));
    cudaError_t e = launch_init_spins(p->L, count, key, init_mode, p->spins + off, st);
    if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    CK(cudaMemsetAsync(p->obs + slot, 0, sizeof(ObsAcc) * count, st));
    CK(cudaMemsetAsync(p->theta2 + (size_t)slot * N, 0, sizeof(double) * N * count, st));
    if (p->hist)
        CK(cudaMemsetAsync(p->hist + (size_t)slot * p->hist_bins, 0,
                           sizeof(unsigned long long) * p->hist_bins * count, st));
    p->last = st;
    if (p->path == MC_PATH_FFT || p->path == MC_PATH_SPECTRAL) {
        // these paths measure the energy afresh; NaN (all bits set) until then,
        // as a lone handle reports before its first measurement
        CK(cudaMemsetAsync(p->energy + slot, 0xFF, sizeof(double) * count, st));
        return MC_OK;
    }
    int rc = anchor_replicas(p, slot, count, st);
    if (rc) return rc;
    p->last = st;
    return MC_OK;
}

void pack_set_sweeps(mc_lattice *p, int slot, int count, int nsweeps) {
    for (int i = 0; i < count; ++i) p->slots_host[slot + i].nsweeps = nsweeps;
}

int pack_launch_direct(mc_lattice *p, int mx, int measure_every, cudaStream_t st);

// Direct packs of one C, proposal, cone and measurement interval in one grouped
// launch (their slots' own counts, as set by pack_set_sweeps); slot counters
// advance as after pack_launch.  *launched = the longest slot's sweeps.
int pack_group_launch(mc_lattice *const *packs, int count, int measure_every, cudaStream_t st, int *launched) {
    int rc = run_group(packs, count, 0, measure_every, st, launched);
    if (rc) return rc;
    for (int i = 0; i < count; ++i) {
        for (SlotState &s : packs[i]->slots_host) {
            s.t0 += (uint32_t)std::max(0, (int)s.nsweeps);
            s.nsweeps = 0;
        }
        packs[i]->last = st;
    }
    return MC_OK;
}

// CTAs a grouped launch of these packs keeps resident at once (0: not groupable).
int pack_group_capacity(mc_lattice *const *packs, int count) {
    int nt = 0, ept = 0;
    size_t smem = 0;
    if (!group_shape(packs, count, &nt, &ept, &smem)) return 0;
    return direct_grouped_resident(packs[0]->L / packs[0]->l, ept, nt, smem);
}

// One packed launch: every slot with nsweeps > 0 advances that many sweeps of its
// own chain; idle slots are untouched.  *launched = the longest slot's sweeps.
int pack_launch(mc_lattice *p, int measure_every, cudaStream_t st, int *launched) {
    *launched = 0;
    int mx = 0;
    for (const SlotState &s : p->slots_host) mx = std::max(mx, (int)s.nsweeps);
    if (mx == 0) return MC_OK;
    CK(cudaEventSynchronize(p->slots_copied));  // the previous launch's staging copy is done
    std::memcpy(p->slots_pin, p->slots_host.data(), sizeof(SlotState) * p->R);
    CK(cudaMemcpyAsync(p->slots_dev, p->slots_pin, sizeof(SlotState) * p->R, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(p->slots_copied, st));
    if (p->path == MC_PATH_FFT || p->path == MC_PATH_SPECTRAL) {
        // these packs replay a captured graph per sweep count; round the count up
        // to a power of two (slots past their own count idle) so that a pack
        // needs only a few graphs
        int g = 1;
        while (g < mx) g <<= 1;
        int rc = run_multi(p, p->path, g, measure_every, nullptr, st);
        if (rc) return rc;
    } else {
        int rc = pack_launch_direct(p, mx, measure_every, st);
        if (rc) return rc;
    }
    for (SlotState &s : p->slots_host) {
        s.t0 += (uint32_t)std::min(mx, (int)s.nsweeps);
        s.nsweeps = 0;
    }
    p->last = st;
    *launched = mx;
    return MC_OK;
}

int pack_launch_direct(mc_lattice *p, int mx, int measure_every, cudaStream_t st) {
    SweepConfig c{};
    c.L = p->L;
    c.l = p->l;
    c.R = p->R;
    c.key = key_of(p->seed);
    c.nsweeps = mx;
    c.measure_every = measure_every;
    c.proposal = p->proposal;
    c.cap_c1 = (float)(1.0 - std::cos(p->cone));
    c.schedule = p->schedule;
    SweepBuffers b;
    b.W32 = p->W32;
    b.spins = p->spins;
    b.params = p->dparams;
    b.energy = p->energy;
    b.obs = p->obs;
    b.theta2 = p->theta2;
    b.slots = p->slots_dev;
    b.hist = hist_of(p);
    cudaError_t e;
    {
        TimedLaunch tl(p, MC_K_SWEEP_DIRECT, st);
        e = launch_sweep_direct(c, b, p->threads_hint, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "packed sweep launch");
    return MC_OK;
}

// Results of replicas [first, first + count): observables and spins [count][3][N]
// to host memory (spins may be null).  Synchronises st.
int read_replicas(mc_lattice *p, int first, int count, cudaStream_t st, mc_obs *obs, float *spins) {
    p->last = st;
    int rc = obs_fill(p, first, count, obs);
    if (rc) return rc;
    if (spins)
        CK(cudaMemcpy(spins, p->spins + (size_t)first * 3 * p->N(), sizeof(float) * 3 * p->N() * count,
                      cudaMemcpyDeviceToHost));
    return MC_OK;
}

// Reuse a lone handle for a new request: new seed, couplings of every replica and
// initial spins, stream-ordered on st (no device-wide synchronisation).
int lattice_refill(mc_lattice *p, uint64_t seed, const RepParams &rp, int init_mode, cudaStream_t st) {
    int rc = check(p);
    if (rc) return rc;
    drop_graphs(p);
    if (!p->params_pin) CK(cudaMallocHost(&p->params_pin, sizeof(RepParams) * p->R));
    for (int i = 0; i < p->R; ++i) p->params_pin[i] = p->hp[i] = rp;
    p->seed = seed;
    CK(cudaMemcpyAsync(p->dparams, p->params_pin, sizeof(RepParams) * p->R, cudaMemcpyHostToDevice, st));
    cudaError_t e = launch_init_spins(p->L, p->R, key_of(seed), init_mode, p->spins, st);
    if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    rc = clear_obs(p, st);
    if (rc) return rc;
    p->t = 0;
    p->energy_valid = false;  // anchored by the first sweep call, on the same stream
    p->last = st;
    return MC_OK;
}

}  // namespace dipmc
