// C ABI of the SIPF-W library: argument checking, device memory of a
// context, and the order of kernel launches of a step (paper Alg. 3).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <dlfcn.h>

#include <algorithm>
#include <utility>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sipf_internal.cuh"

namespace {

using namespace sipf;

int fail(sipf_ctx* c, int code, const std::string& msg) {
    if (c) c->last_error = msg;
    return code;
}

int cuda_fail(sipf_ctx* c, cudaError_t e, const char* where) {
    return fail(c, SIPF_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define SIPF_CUDA(ctx, call)                                         \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);   \
    } while (0)

// Grid sides with a radix plan (2^a 3^b) that are multiples of the 8-cell tile.
// ---------------------------------------------------------------- tuning table
// Process-wide table of tuning choices by grid size and particle count,
// read from a text file (the autotuner writes it): lines
//   H  N_min  N_max  radix_plan  step_blocks_per_sm  bucket_slack_div  bucket_slack_add
// ('#' starts a comment).  The first matching line applies to a new context.
struct TuneEntry {
    int H;
    int64_t n_min, n_max;
    sipf_tuning t;
};
std::mutex g_tune_mutex;
std::vector<TuneEntry> g_tune;
bool g_tune_loaded = false;

bool tuning_valid(const sipf_tuning& t) {
    return t.radix_plan >= 0 && t.radix_plan <= 2 && t.step_blocks_per_sm >= 0 &&
           t.step_blocks_per_sm <= 32 && t.bucket_slack_div >= 8 &&
           t.bucket_slack_div <= 1024 && t.bucket_slack_add >= 0 && t.bucket_slack_add <= 32;
}

int parse_tuning_file(const char* path, std::vector<TuneEntry>* out) {
    FILE* f = fopen(path, "r");
    if (!f) return SIPF_EINVAL;
    char line[512];
    int rc = SIPF_OK;
    while (fgets(line, sizeof line, f)) {
        char* hash = strchr(line, '#');
        if (hash) *hash = 0;
        TuneEntry e{};
        long long lo = 0, hi = 0;
        const int got = sscanf(line, "%d %lld %lld %d %d %d %d", &e.H, &lo, &hi, &e.t.radix_plan,
                               &e.t.step_blocks_per_sm, &e.t.bucket_slack_div,
                               &e.t.bucket_slack_add);
        if (got <= 0) continue;   // blank or comment
        e.n_min = lo;
        e.n_max = hi;
        if (got != 7 || !tuning_valid(e.t) || lo > hi) {
            rc = SIPF_EINVAL;
            break;
        }
        out->push_back(e);
    }
    fclose(f);
    return rc;
}

// The table next to the library (sipf_tuning.txt in the directory of
// libsipf.so), or the file named by SIPF_TUNING, read on first use.
void load_default_tuning_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    std::string path;
    if (const char* env = getenv("SIPF_TUNING")) {
        path = env;
    } else {
        Dl_info info;
        if (dladdr(reinterpret_cast<void*>(&load_default_tuning_locked), &info) && info.dli_fname) {
            path = info.dli_fname;
            const size_t slash = path.rfind('/');
            path = (slash == std::string::npos ? std::string(".") : path.substr(0, slash)) +
                   "/sipf_tuning.txt";
        }
    }
    std::vector<TuneEntry> t;
    if (!path.empty() && parse_tuning_file(path.c_str(), &t) == SIPF_OK) g_tune = t;
}

bool lookup_tuning(int H, int64_t N, sipf_tuning* out) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    load_default_tuning_locked();
    for (const TuneEntry& e : g_tune)
        if (e.H == H && N >= e.n_min && N <= e.n_max) {
            *out = e.t;
            return true;
        }
    return false;
}

void apply_tuning(sipf_ctx* c, const sipf_tuning& t) {
    // plan 2 (the warp pipeline) where the grid size has it, else plan 0
    c->radix_plan = t.radix_plan == 2 && !has_warp_pipeline(c->H) ? 0 : t.radix_plan;
    c->step_bps = t.step_blocks_per_sm;
    c->slack_div = t.bucket_slack_div;
    c->slack_add = t.bucket_slack_add;
}

bool supported_H(int H) {
    switch (H) {
        case 8: case 16: case 24: case 32: case 48: case 64: case 72: case 96: case 128:
        case 144: case 192: case 216: case 256: case 288: case 384: case 432: case 512:
            return true;
        default:
            return false;
    }
}

bool finite_nonneg(double x) { return isfinite(x) && x >= 0.0; }

int check_params(const sipf_params* p, std::string* why) {
    const double v[] = {p->chi, p->Du, p->Dm, p->Dw, p->alpha, p->beta, p->gamma, p->H0, p->sigma};
    const char* n[] = {"chi", "Du", "Dm", "Dw", "alpha", "beta", "gamma", "H0", "sigma"};
    for (int i = 0; i < 9; ++i)
        if (!finite_nonneg(v[i])) {
            *why = std::string("parameter ") + n[i] + " must be finite and >= 0";
            return SIPF_EINVAL;
        }
    if (p->diffusion != SIPF_DIFFUSION_IMPLICIT && p->diffusion != SIPF_DIFFUSION_EXP) {
        *why = "unknown diffusion mode";
        return SIPF_EINVAL;
    }
    if (p->v_update != SIPF_V_IMPLICIT && p->v_update != SIPF_V_EXPLICIT) {
        *why = "unknown v_update mode";
        return SIPF_EINVAL;
    }
    if ((p->p2g_order != 0 && p->p2g_order != 2 && p->p2g_order != 4) || p->reserved != 0) {
        *why = "p2g_order must be 0, 2 or 4 (and reserved 0)";
        return SIPF_EINVAL;
    }
    return SIPF_OK;
}

template <class T>
cudaError_t dalloc(T** p, size_t n) {
    return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

// Sizes of a context's device arrays (shared by sipf_create and the memory
// estimate sipf_context_bytes).
struct CtxSizes {
    size_t H3, spec;
    int ntiles, ovf_base, max_items;
    int64_t buf_slots;
};

CtxSizes ctx_sizes(int H, int64_t N) {
    CtxSizes z;
    z.H3 = static_cast<size_t>(H) * H * H;
    z.spec = static_cast<size_t>(H) * H * (H / 2 + 2);
    const int T = H / 8;
    z.ntiles = T * T * T;
    const int64_t bucket_slots = N + N / 8 + 36 * static_cast<int64_t>(z.ntiles) + 64;
    z.ovf_base = static_cast<int>((bucket_slots + 3) & ~int64_t{3});
    z.buf_slots = z.ovf_base + N + 8;
    const int K = item_size();
    z.max_items = static_cast<int>(2 * ((N + K - 1) / K) + z.ntiles + 2);
    return z;
}

// Device bytes sipf_create allocates (the resampling work space, allocated
// on first use, is not included).
size_t ctx_device_bytes(int H, int64_t N, bool filter, bool smoothing) {
    const CtxSizes z = ctx_sizes(H, N);
    const size_t S = static_cast<size_t>(z.buf_slots);
    size_t b = 2 * (S * (3 * sizeof(float) + sizeof(double) + sizeof(uint32_t)) +
                    3 * static_cast<size_t>(z.ntiles) * sizeof(int) + sizeof(int));
    b += static_cast<size_t>(z.max_items) * sizeof(Item) + 2 * sizeof(int);
    b += z.H3 * sizeof(int32_t) + (z.H3 + 1) * sizeof(int32_t) +
         (static_cast<size_t>(scan_tiles(static_cast<int>(z.H3))) + 1) * sizeof(int32_t);
    b += z.H3 * sizeof(long long) + 3 * z.H3 * sizeof(float) + 4 * z.H3 * sizeof(float);
    b += 4 * z.spec * sizeof(float2) + static_cast<size_t>(H) * sizeof(float2);
    b += sizeof(int) + sizeof(float) + 2 * sizeof(StepScalars);
    b += diag_scratch_doubles() * sizeof(double) + diag_scratch_ll() * sizeof(long long) +
         8 * sizeof(double);
    if (filter) b += z.spec * sizeof(float2);
    if (H > 128 || has_warp_pipeline(H)) b += 2 * z.spec * sizeof(float2);
    if (smoothing) b += z.H3 * sizeof(float) + static_cast<size_t>(H) * sizeof(float);
    return b;
}

// Frees the arrays sipf_create allocated (stream-ordered on the context's
// stream when they came from a pool) and the resampling work space.
void free_all(sipf_ctx* c) {
    void* ptrs[] = {c->sx[0], c->sx[1], c->sy[0], c->sy[1], c->sz[0], c->sz[1], c->dl[0],
                    c->dl[1], c->id[0], c->id[1], c->bstart[0], c->bstart[1], c->cap[0],
                    c->cap[1], c->cnt[0], c->cnt[1], c->ovf[0], c->ovf[1], c->items, c->n_items,
                    c->work, c->count, c->cell_start, c->scan_tmp, c->acc, c->v, c->m, c->w,
                    c->G, c->specM, c->specW, c->specV, c->specB, c->specA, c->specDx,
                    c->specDy, c->twiddle,
                    c->status, c->diag_tmp, c->diag_out, c->diag_ll, c->voff,
                    c->dsc, c->us, c->ksig};
    for (void* q : ptrs) {
        if (!q) continue;
        if (c->pool)
            cudaFreeAsync(q, c->stream);
        else
            cudaFree(q);
    }
    if (c->rs_scratch) cudaFree(c->rs_scratch);
}

int copy_in(sipf_ctx* c, void* dst, const void* src, size_t bytes, int where) {
    const cudaMemcpyKind k = where == SIPF_DEVICE ? cudaMemcpyDeviceToDevice
                                                  : cudaMemcpyHostToDevice;
    SIPF_CUDA(c, cudaMemcpyAsync(dst, src, bytes, k, c->stream));
    return SIPF_OK;
}

int copy_out(sipf_ctx* c, void* dst, const void* src, size_t bytes, int where) {
    const cudaMemcpyKind k = where == SIPF_DEVICE ? cudaMemcpyDeviceToDevice
                                                  : cudaMemcpyDeviceToHost;
    SIPF_CUDA(c, cudaMemcpyAsync(dst, src, bytes, k, c->stream));
    return SIPF_OK;
}

int check_status(sipf_ctx* c) {
    int st = 0;
    SIPF_CUDA(c, cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SIPF_CUDA(c, cudaStreamSynchronize(c->stream));
    if (st) {
        SIPF_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
        if (st & kStatusNonfinite)
            return fail(c, SIPF_ENONFINITE, "a particle position became non-finite and was reset");
        return fail(c, SIPF_EINTERNAL,
                    std::string("device consistency check failed (status ") +
                        std::to_string(st) + ")");
    }
    return SIPF_OK;
}

// Fixed-point scale 2^S of the deposit at the context's current time (the
// same expression the plan kernel evaluates for the device-side scalars).
int deposit_shift(const sipf_ctx* c) { return deposit_shift_at(c->log2_maxrel, c->time); }

// Converts the integer accumulator to u_bar = a R_h summed: 2^-S e^logref / h^3.
double acc_to_u_d(const sipf_ctx* c) { return ldexp(c->exp_logref, -deposit_shift(c)) / c->h3; }

float acc_to_u(const sipf_ctx* c) { return static_cast<float>(acc_to_u_d(c)); }

// The device scalars of the next step (slot of the current buffer) from the
// host's step count and time; after set-up operations that do not advance a
// step (set_state, load, resample).
int write_scalars(sipf_ctx* c) {
    StepScalars hs;
    fill_step_scalars(&hs, static_cast<uint32_t>(c->step + 1), c->time, c->log2_maxrel,
                      c->exp_logref, c->h3);
    SIPF_CUDA(c, cudaMemcpyAsync(c->dsc + c->cur, &hs, sizeof(hs), cudaMemcpyHostToDevice,
                                 c->stream));
    SIPF_CUDA(c, cudaStreamSynchronize(c->stream));
    return SIPF_OK;
}

// Constants of the scalars from logref and maxrel.
void set_mass_reference(sipf_ctx* c) {
    c->log2_maxrel = log2(c->maxrel);
    c->exp_logref = exp(c->logref);
}

PushArgs push_args(const sipf_ctx* c, double dt, int push) {
    PushArgs a;
    a.H = c->H;
    a.drift = static_cast<float>(c->p.chi * dt / c->h);
    a.noise = static_cast<float>(sqrt(2.0 * c->p.Du * dt) / c->h);
    a.tau = static_cast<float>(dt);
    a.k0 = static_cast<uint32_t>(c->p.seed);
    a.k1 = static_cast<uint32_t>(c->p.seed >> 32);
    for (int r = 0; r < 10; ++r) {
        a.rk[2 * r] = a.k0 + static_cast<uint32_t>(r) * 0x9E3779B9u;
        a.rk[2 * r + 1] = a.k1 + static_cast<uint32_t>(r) * 0xBB67AE85u;
    }
    a.push = push;
    return a;
}

SpectralArgs spectral_args(const sipf_ctx* c, double dt, int full) {
    SpectralArgs s;
    s.tau = static_cast<float>(dt);
    s.gamma = static_cast<float>(c->p.gamma);
    s.alpha = static_cast<float>(c->p.alpha);
    s.v_update = c->p.v_update;
    s.diffusion = c->p.diffusion;
    s.two_pi_over_L = static_cast<float>(2.0 * M_PI / c->L);
    const double k1 = (2.0 * M_PI / c->L) * (2.0 * M_PI / c->L);
    const double R[2] = {c->p.beta, 1.0}, D[2] = {c->p.Dm, c->p.Dw};
    float* hi[2] = {&s.m_r0_hi, &s.w_r0_hi};
    float* lo[2] = {&s.m_r0_lo, &s.w_r0_lo};
    float* cc[2] = {&s.m_c, &s.w_c};
    for (int f = 0; f < 2; ++f) {
        const bool impl = c->p.diffusion == SIPF_DIFFUSION_IMPLICIT;
        const double r0 = impl ? 1.0 / (1.0 + dt * R[f]) : exp(-dt * R[f]);
        *hi[f] = static_cast<float>(r0);
        *lo[f] = static_cast<float>(r0 - static_cast<double>(*hi[f]));
        *cc[f] = static_cast<float>(impl ? dt * D[f] * k1 * r0 : dt * D[f] * k1);
    }
    s.filter = (c->p.H0 > 0.0 && c->p.H0 < c->H) ? 1 : 0;
    s.inv_H0sq_2pi2 = s.filter ? static_cast<float>(2.0 * M_PI * M_PI / (c->p.H0 * c->p.H0)) : 0.f;
    s.out_scale = static_cast<float>(1.0 / (static_cast<double>(c->H) * c->H * c->H));
    // without the filter the v spectrum used for dv/dx, dv/dy is never
    // transformed along z, so its inverse carries H^2 instead of H^3
    s.out_scale_xy = s.filter ? s.out_scale
                              : static_cast<float>(1.0 / (static_cast<double>(c->H) * c->H));
    s.write_v = full;
    s.do_mw = full;
    return s;
}

// Bin the unbinned particles of buffer b (slots [0, N)) into tile buckets of
// buffer b ^ 1, and plan the items of b ^ 1 and the layout of b.
int bin_from(sipf_ctx* c, int b) {
    SIPF_CUDA(c, cudaMemsetAsync(c->cnt[b], 0, sizeof(int) * c->ntiles, c->stream));
    SIPF_CUDA(c, cudaMemsetAsync(c->ovf[b], 0, sizeof(int), c->stream));
    SIPF_CUDA(c, launch_tile_count(c, b, c->cnt[b]));
    SIPF_CUDA(c, launch_plan(c, b, 1, c->stream, 0.0));   // layout of buffer b ^ 1 from the tile counts
    SIPF_CUDA(c, launch_plan_flat(c));           // items: the raw input array
    c->cur = b;
    const PushArgs a = push_args(c, 0.0, 0);
    SIPF_CUDA(c, launch_step_kernel(c, a, 0, 1));
    c->cur = b ^ 1;
    SIPF_CUDA(c, launch_plan(c, b ^ 1, 1, c->stream, 0.0));
    return SIPF_OK;
}

int bin_initial(sipf_ctx* c) { return bin_from(c, 1); }

// Deposit the current particles into the accumulator (Alg. 1).
int deposit_current(sipf_ctx* c) {
    const PushArgs a = push_args(c, 0.0, 0);
    SIPF_CUDA(c, launch_step_kernel(c, a, 1, 0));
    return SIPF_OK;
}

// Compact the live particles of the current buffer into the other buffer
// (slots [0, N), item order), which is free between steps.
int compact_current(sipf_ctx* c) {
    SIPF_CUDA(c, launch_compact(c, c->cur, c->cur ^ 1));
    return SIPF_OK;
}

// Event k of the current step (tracing); nullptr when not recording.
cudaEvent_t prof_event(sipf_ctx* c, int k) {
    if (!c->prof_on || c->prof_steps >= kProfMaxSteps) return nullptr;
    const size_t i = static_cast<size_t>(c->prof_steps) * (kProfGroups + 1) + k;
    while (c->prof_events.size() <= i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->prof_events.push_back(e);
    }
    return c->prof_events[i];
}

cudaError_t prof_mark(sipf_ctx* c, int k) {
    cudaEvent_t e = prof_event(c, k);
    return e ? cudaEventRecord(e, c->stream) : cudaSuccess;
}

// Host bookkeeping of one step (the device side advances its scalars in the
// plan kernel).
void advance_host(sipf_ctx* c, double dt) {
    c->cur ^= 1;
    c->step += 1;
    c->time += dt;
}

int enqueue_step(sipf_ctx* c, double dt) {
    const PushArgs a = push_args(c, dt, 1);
    const SpectralArgs sa = spectral_args(c, dt, 1);
    SIPF_CUDA(c, prof_mark(c, 0));
    SIPF_CUDA(c, launch_step_kernel(c, a, 1, 1));
    SIPF_CUDA(c, prof_mark(c, 1));
    // the plan of the next step's items, layout and scalars needs only the
    // counts: it runs on the side stream while the spectral passes run on the main one
    SIPF_CUDA(c, cudaEventRecord(c->ev_fork, c->stream));
    SIPF_CUDA(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    SIPF_CUDA(c, launch_plan(c, c->cur ^ 1, 1, c->side, dt));
    SIPF_CUDA(c, cudaEventRecord(c->ev_join, c->side));
    // K_sigma * u_bar for the m source (Eq. m_reg), when sigma > 0
    if (c->us) SIPF_CUDA(c, launch_smooth(c, c->us, c->stream));
    for (int pass = 0; pass < 3; ++pass) {
        SIPF_CUDA(c, launch_spectral_pass(c, sa, pass));
        SIPF_CUDA(c, prof_mark(c, 2 + pass));
    }
    SIPF_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    if (c->prof_on && c->prof_steps < kProfMaxSteps) c->prof_steps += 1;
    advance_host(c, dt);
    return SIPF_OK;
}

// Two steps of size dt captured once (per dt and buffer parity) as a CUDA
// graph; *out = nullptr when the stream cannot capture (the legacy default
// stream) or capture fails, in which case the caller enqueues the steps.
int step_pair_graph(sipf_ctx* c, double dt, cudaGraphExec_t* out) {
    *out = nullptr;
    if (!c->stream) return SIPF_OK;
    for (const auto& g : c->graphs)
        if (g.dt == dt && g.parity == c->cur) {
            *out = g.exec;
            return SIPF_OK;
        }
    const int cur0 = c->cur;
    const int64_t step0 = c->step;
    const double time0 = c->time;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return SIPF_OK;
    }
    int r = enqueue_step(c, dt);
    if (r == SIPF_OK) r = enqueue_step(c, dt);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    c->cur = cur0;
    c->step = step0;
    c->time = time0;
    cudaGraphExec_t exec = nullptr;
    const bool ok = r == SIPF_OK && e == cudaSuccess && graph &&
                    cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        return SIPF_OK;
    }
    if (c->graphs.size() >= 4) {
        cudaGraphExecDestroy(c->graphs.front().exec);
        c->graphs.erase(c->graphs.begin());
    }
    c->graphs.push_back({dt, cur0, exec});
    *out = exec;
    return SIPF_OK;
}

// k steps: pairs replay the captured two-step graph (not while tracing),
// the rest is enqueued launch by launch; both run the same kernels with the
// same arguments.
int run_steps(sipf_ctx* c, double dt, int64_t k) {
    int64_t done = 0;
    if (k >= 2 && !c->prof_on) {
        cudaGraphExec_t exec = nullptr;
        const int r = step_pair_graph(c, dt, &exec);
        if (r != SIPF_OK) return r;
        for (; exec && done + 2 <= k; done += 2) {
            SIPF_CUDA(c, cudaGraphLaunch(exec, c->stream));
            advance_host(c, dt);
            advance_host(c, dt);
        }
    }
    for (; done < k; ++done) {
        const int r = enqueue_step(c, dt);
        if (r != SIPF_OK) return r;
    }
    return SIPF_OK;
}

// ---------------------------------------------------------------- checkpoints
// File layout (native byte order): CkptHeader, then the payload arrays in
// the order sx, sy, sz (N float, grid units), dl (N double, log a - logref),
// id (N uint32), v, m, w (H^3 float), G (4 H^3 float).
constexpr char kCkptMagic[8] = {'S', 'I', 'P', 'F', 'C', 'K', 'P', 'T'};
constexpr uint32_t kCkptVersion = 1;

struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;   // sizeof(CkptHeader)
    int32_t H;
    int32_t pad0;
    double L;
    double origin[3];
    int64_t N;
    sipf_params params;
    int64_t step;
    double time;
    double logref;
    double maxrel;
    float voff;
    uint32_t pad1;
    uint64_t payload_bytes;
    uint64_t payload_hash;   // ckpt_hash of the payload
};

// 64-bit FNV-1a over 8-byte words (a final partial word is zero-padded).
uint64_t ckpt_hash(uint64_t h, const void* data, size_t bytes) {
    const unsigned char* b = static_cast<const unsigned char*>(data);
    size_t i = 0;
    for (; i + 8 <= bytes; i += 8) {
        uint64_t w;
        memcpy(&w, b + i, 8);
        h = (h ^ w) * 0x100000001B3ull;
    }
    if (i < bytes) {
        uint64_t w = 0;
        memcpy(&w, b + i, bytes - i);
        h = (h ^ w) * 0x100000001B3ull;
    }
    return h;
}

struct CkptArray {
    void* dev;
    size_t bytes;
};

}  // namespace

namespace sipf {
// k steps of a context with the same launch path as sipf_step (graph pairs
// when possible), for the request scheduler.
int run_steps_for(sipf_ctx* c, double dt, int64_t k) { return run_steps(c, dt, k); }
}  // namespace sipf

extern "C" {

const char* sipf_strerror(int code) {
    switch (code) {
        case SIPF_OK: return "success";
        case SIPF_EINVAL: return "invalid argument";
        case SIPF_ENOMEM: return "out of memory";
        case SIPF_ECUDA: return "CUDA error";
        case SIPF_EUNSUPPORTED: return "unsupported configuration";
        case SIPF_ENONFINITE: return "non-finite particle position";
        case SIPF_EINTERNAL: return "device consistency check failed";
        default: return "unknown error";
    }
}

const char* sipf_last_error(const sipf_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int sipf_create(const sipf_grid* grid, int64_t N, const sipf_params* params, void* stream,
                sipf_ctx** out) {
    return sipf::create_in_pool(grid, N, params, static_cast<cudaStream_t>(stream), nullptr, out);
}

}  // extern "C"

namespace sipf {

int create_in_pool(const sipf_grid* grid, int64_t N, const sipf_params* params,
                   cudaStream_t stream, cudaMemPool_t pool, sipf_ctx** out) {
    if (!out || !grid || !params) return SIPF_EINVAL;
    *out = nullptr;
    std::string why;
    if (N < 1 || N >= (int64_t{1} << 31)) return SIPF_EINVAL;
    if (!(isfinite(grid->L) && grid->L > 0.0)) return SIPF_EINVAL;
    for (int k = 0; k < 3; ++k)
        if (!isfinite(grid->origin[k])) return SIPF_EINVAL;
    if (!supported_H(grid->H)) return SIPF_EINVAL;
    if (check_params(params, &why) != SIPF_OK) return SIPF_EINVAL;

    sipf_ctx* c = new (std::nothrow) sipf_ctx();
    if (!c) return SIPF_ENOMEM;
    c->H = grid->H;
    c->L = grid->L;
    c->h = grid->L / grid->H;
    c->h3 = c->h * c->h * c->h;
    for (int k = 0; k < 3; ++k) c->origin[k] = grid->origin[k];
    c->N = N;
    c->p = *params;
    if (c->p.p2g_order == 0) c->p.p2g_order = 2;
    c->stream = stream;
    c->pool = pool;
    cudaGetDevice(&c->device);
    const CtxSizes z = ctx_sizes(c->H, N);
    const size_t H3 = z.H3, spec = z.spec;
    c->kxp = c->H / 2 + 2;
    c->ntiles = z.ntiles;
    c->ovf_base = z.ovf_base;
    c->buf_slots = z.buf_slots;
    if (c->buf_slots >= (int64_t{1} << 31)) {
        delete c;
        return SIPF_EINVAL;
    }
    c->max_items = z.max_items;
    const size_t S = static_cast<size_t>(c->buf_slots);
    // every allocation of the context is counted in dev_bytes
    auto da = [c](auto** p, size_t n) {
        c->dev_bytes += n * sizeof(**p);
        if (c->pool)
            return cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), n * sizeof(**p), c->pool,
                                           c->stream);
        return dalloc(p, n);
    };
    bool ok = true;
    for (int b = 0; b < 2; ++b) {
        ok = ok && da(&c->sx[b], S) == cudaSuccess && da(&c->sy[b], S) == cudaSuccess &&
             da(&c->sz[b], S) == cudaSuccess && da(&c->dl[b], S) == cudaSuccess &&
             da(&c->id[b], S) == cudaSuccess &&
             da(&c->bstart[b], c->ntiles) == cudaSuccess &&
             da(&c->cap[b], c->ntiles) == cudaSuccess &&
             da(&c->cnt[b], c->ntiles) == cudaSuccess && da(&c->ovf[b], 1) == cudaSuccess;
    }
    ok = ok && da(&c->items, static_cast<size_t>(c->max_items)) == cudaSuccess &&
         da(&c->n_items, 1) == cudaSuccess && da(&c->work, 1) == cudaSuccess &&
         da(&c->count, H3) == cudaSuccess && da(&c->cell_start, H3 + 1) == cudaSuccess &&
         da(&c->scan_tmp, static_cast<size_t>(scan_tiles(static_cast<int>(H3))) + 1) == cudaSuccess &&
         da(&c->acc, H3) == cudaSuccess && da(&c->v, H3) == cudaSuccess &&
         da(&c->m, H3) == cudaSuccess && da(&c->w, H3) == cudaSuccess &&
         da(&c->G, 4 * H3) == cudaSuccess && da(&c->specM, spec) == cudaSuccess &&
         da(&c->specW, spec) == cudaSuccess && da(&c->specV, spec) == cudaSuccess &&
         da(&c->specB, spec) == cudaSuccess && da(&c->twiddle, c->H) == cudaSuccess &&
         da(&c->status, 1) == cudaSuccess && da(&c->voff, 1) == cudaSuccess &&
         da(&c->dsc, 2) == cudaSuccess &&
         da(&c->diag_tmp, diag_scratch_doubles()) == cudaSuccess &&
         da(&c->diag_ll, diag_scratch_ll()) == cudaSuccess &&
         da(&c->diag_out, 8) == cudaSuccess;
    const bool filter = params->H0 > 0.0 && params->H0 < grid->H;
    if (ok && filter) ok = da(&c->specA, spec) == cudaSuccess;
    if (ok && (c->H > 128 || has_warp_pipeline(c->H)))
        ok = da(&c->specDx, spec) == cudaSuccess && da(&c->specDy, spec) == cudaSuccess;
    if (ok && params->sigma > 0.0)
        ok = da(&c->us, H3) == cudaSuccess && da(&c->ksig, static_cast<size_t>(c->H)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return SIPF_ENOMEM;
    }
    // host staging lives until the stream synchronisation below
    std::vector<float2> tw(c->H);
    std::vector<float> ks(c->ksig ? c->H : 0);
    fill_twiddles(c->H, tw.data());
    cudaError_t e = cudaMemcpyAsync(c->twiddle, tw.data(), c->H * sizeof(float2),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && c->ksig) {
        fill_smoothing(c->H, c->L, params->sigma, ks.data());
        e = cudaMemcpyAsync(c->ksig, ks.data(), c->H * sizeof(float), cudaMemcpyHostToDevice,
                            c->stream);
    }
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaMemsetAsync(c->bstart[b], 0, sizeof(int) * c->ntiles, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->cap[b], 0, sizeof(int) * c->ntiles, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->cnt[b], 0, sizeof(int) * c->ntiles, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->ovf[b], 0, sizeof(int), c->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->acc, 0, H3 * sizeof(long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->G, 0, 4 * H3 * sizeof(float), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dsc, 0, 2 * sizeof(StepScalars), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return SIPF_ECUDA;
    }
    sipf_tuning tuned;
    if (lookup_tuning(c->H, N, &tuned)) apply_tuning(c, tuned);
    c->step_blocks = step_grid(c);
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        free_all(c);
        delete c;
        return SIPF_ECUDA;
    }
    *out = c;
    return SIPF_OK;
}

}  // namespace sipf

extern "C" {

int sipf_set_state(sipf_ctx* c, const float* x, const double* mass, const uint32_t* id,
                   const float* v, const float* m, const float* w, int where) {
    if (!c) return SIPF_EINVAL;
    if (!x || !mass || !v || !m || !w) return fail(c, SIPF_EINVAL, "NULL input pointer");
    if (where != SIPF_HOST && where != SIPF_DEVICE) return fail(c, SIPF_EINVAL, "bad where");
    const size_t N = static_cast<size_t>(c->N);
    const size_t H3 = static_cast<size_t>(c->H) * c->H * c->H;
    // reference log-mass logref = log(M0 / N) from the masses (host FP64 sum)
    std::vector<double> hm;
    const double* mp = mass;
    if (where == SIPF_DEVICE) {
        hm.resize(N);
        SIPF_CUDA(c, cudaMemcpyAsync(hm.data(), mass, N * sizeof(double), cudaMemcpyDeviceToHost,
                                     c->stream));
        SIPF_CUDA(c, cudaStreamSynchronize(c->stream));
        mp = hm.data();
    }
    double M0 = 0.0, amax = 0.0;
    for (size_t i = 0; i < N; ++i) {
        if (!(isfinite(mp[i]) && mp[i] >= 0.0))
            return fail(c, SIPF_EINVAL, "masses must be finite and >= 0");
        M0 += mp[i];
        amax = mp[i] > amax ? mp[i] : amax;
    }
    c->logref = M0 > 0.0 ? log(M0 / static_cast<double>(N)) : 0.0;
    c->maxrel = M0 > 0.0 ? amax / exp(c->logref) : 1.0;
    set_mass_reference(c);
    c->step = 0;
    c->time = 0.0;
    // wrap into buffer 1 (unordered), then bin into buffer 0.  Host input is
    // staged in buffer 0 first (free until the binning; each of its arrays
    // has room for N values), so the call allocates nothing.
    const float* px = x;
    const float* py = x + N;
    const float* pz = x + 2 * N;
    const double* pm = mass;
    if (where == SIPF_HOST) {
        int r = copy_in(c, c->sx[0], x, N * sizeof(float), SIPF_HOST);
        if (r == SIPF_OK) r = copy_in(c, c->sy[0], x + N, N * sizeof(float), SIPF_HOST);
        if (r == SIPF_OK) r = copy_in(c, c->sz[0], x + 2 * N, N * sizeof(float), SIPF_HOST);
        if (r == SIPF_OK) r = copy_in(c, c->dl[0], mass, N * sizeof(double), SIPF_HOST);
        if (r != SIPF_OK) return r;
        px = c->sx[0];
        py = c->sy[0];
        pz = c->sz[0];
        pm = c->dl[0];
    }
    int r = SIPF_OK;
    cudaError_t e = launch_wrap_positions(c, px, py, pz, 1);
    if (e == cudaSuccess) e = launch_rel_log_mass(c, pm, 1);
    if (e == cudaSuccess) {
        if (id) {
            r = copy_in(c, c->id[1], id, N * sizeof(uint32_t), where);
        } else {
            e = launch_iota(c, 1);
        }
    }
    if (e == cudaSuccess && r == SIPF_OK) {
        // offset for the v transform: the mean of v^(0) (only derivatives of
        // the v spectrum are used, so any constant may be removed first)
        std::vector<float> hv;
        const float* vp = v;
        if (where == SIPF_DEVICE) {
            hv.resize(H3);
            e = cudaMemcpyAsync(hv.data(), v, H3 * sizeof(float), cudaMemcpyDeviceToHost,
                                c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            vp = hv.data();
        }
        double vs = 0.0;
        for (size_t i = 0; e == cudaSuccess && i < H3; ++i) vs += vp[i];
        c->voff_host = static_cast<float>(vs / static_cast<double>(H3));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->voff, &c->voff_host, sizeof(float), cudaMemcpyHostToDevice,
                                c->stream);
    }
    if (e == cudaSuccess && r == SIPF_OK) {
        r = copy_in(c, c->v, v, H3 * sizeof(float), where);
        if (r == SIPF_OK) r = copy_in(c, c->m, m, H3 * sizeof(float), where);
        if (r == SIPF_OK) r = copy_in(c, c->w, w, H3 * sizeof(float), where);
    }
    if (e == cudaSuccess && r == SIPF_OK) r = bin_initial(c);
    if (e == cudaSuccess && r == SIPF_OK) {
        // w^(0) into the gather array; grad v^(0) from the DFT of v^(0) (tau = 0)
        e = cudaMemcpy2DAsync(c->G + 3, 4 * sizeof(float), c->w, sizeof(float), sizeof(float), H3,
                              cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = launch_spectral_step(c, spectral_args(c, 0.0, 0));
    }
    if (e == cudaSuccess && r == SIPF_OK) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "sipf_set_state");
    if (r != SIPF_OK) return r;
    r = check_status(c);
    if (r != SIPF_OK) return r;
    r = write_scalars(c);
    if (r != SIPF_OK) return r;
    c->state_set = true;
    return SIPF_OK;
}

int sipf_step(sipf_ctx* c, double dt, int64_t k) {
    if (!c) return SIPF_EINVAL;
    if (!c->state_set) return fail(c, SIPF_EINVAL, "sipf_set_state has not been called");
    if (!(isfinite(dt) && dt > 0.0 && dt <= 0.5))
        return fail(c, SIPF_EINVAL, "dt must satisfy 0 < dt <= 0.5");
    if (k < 0) return fail(c, SIPF_EINVAL, "k must be >= 0");
    return run_steps(c, dt, k);
}

int sipf_fields(sipf_ctx* c, uint32_t mask, float* dst, int where) {
    if (!c) return SIPF_EINVAL;
    if (!dst || (mask & ~127u)) return fail(c, SIPF_EINVAL, "bad dst or mask");
    if (where != SIPF_HOST && where != SIPF_DEVICE) return fail(c, SIPF_EINVAL, "bad where");
    if (!c->state_set) return fail(c, SIPF_EINVAL, "sipf_set_state has not been called");
    const size_t H3 = static_cast<size_t>(c->H) * c->H * c->H;
    const float* src[4] = {nullptr, c->v, c->m, c->w};
    // staging for host copies: the per-cell histogram array (H^3 words, used
    // only by sipf_cell_start), so the call allocates nothing
    float* tmp = reinterpret_cast<float*>(c->count);
    size_t off = 0;
    for (int b = 0; b < 7; ++b) {
        if (!(mask & (1u << b))) continue;
        if (b >= 4) {
            if (where == SIPF_DEVICE) {
                SIPF_CUDA(c, launch_component(c, b - 4, dst + off));
            } else {
                cudaError_t e = launch_component(c, b - 4, tmp);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(dst + off, tmp, H3 * sizeof(float), cudaMemcpyDeviceToHost,
                                        c->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                if (e != cudaSuccess) return cuda_fail(c, e, "sipf_fields(grad v)");
            }
        } else if (b == 0) {
            int r = deposit_current(c);
            if (r != SIPF_OK) return r;
            if (where == SIPF_DEVICE) {
                SIPF_CUDA(c, launch_acc_to_float(c, dst + off, acc_to_u(c)));
            } else {
                cudaError_t e = launch_acc_to_float(c, tmp, acc_to_u(c));
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(dst + off, tmp, H3 * sizeof(float), cudaMemcpyDeviceToHost,
                                        c->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                if (e != cudaSuccess) return cuda_fail(c, e, "sipf_fields(U)");
            }
        } else {
            int r = copy_out(c, dst + off, src[b], H3 * sizeof(float), where);
            if (r != SIPF_OK) return r;
        }
        off += H3;
    }
    return check_status(c);
}

int sipf_particle_state(sipf_ctx* c, float* s, double* loga, uint32_t* id, int where) {
    if (!c) return SIPF_EINVAL;
    if (where != SIPF_HOST && where != SIPF_DEVICE) return fail(c, SIPF_EINVAL, "bad where");
    if (!c->state_set) return fail(c, SIPF_EINVAL, "sipf_set_state has not been called");
    const size_t N = static_cast<size_t>(c->N);
    int r = compact_current(c);
    const int o = c->cur ^ 1;
    if (r == SIPF_OK && s) {
        r = copy_out(c, s, c->sx[o], N * sizeof(float), where);
        if (r == SIPF_OK) r = copy_out(c, s + N, c->sy[o], N * sizeof(float), where);
        if (r == SIPF_OK) r = copy_out(c, s + 2 * N, c->sz[o], N * sizeof(float), where);
    }
    if (r == SIPF_OK && loga) {
        // log a = dl + logref, in place in the free buffer
        SIPF_CUDA(c, launch_export_mass(c, o, c->dl[o], 1));
        r = copy_out(c, loga, c->dl[o], N * sizeof(double), where);
    }
    if (r == SIPF_OK && id) r = copy_out(c, id, c->id[o], N * sizeof(uint32_t), where);
    if (r != SIPF_OK) return r;
    return check_status(c);
}

int sipf_particles(sipf_ctx* c, float* x, double* mass, uint32_t* id, int where) {
    if (!c) return SIPF_EINVAL;
    if (where != SIPF_HOST && where != SIPF_DEVICE) return fail(c, SIPF_EINVAL, "bad where");
    if (!c->state_set) return fail(c, SIPF_EINVAL, "sipf_set_state has not been called");
    const size_t N = static_cast<size_t>(c->N);
    int r = compact_current(c);
    if (r != SIPF_OK) return r;
    const int o = c->cur ^ 1;
    // the compacted copy in the free buffer is converted in place (positions
    // to physical coordinates, log-masses to masses), so nothing is allocated
    cudaError_t e = cudaSuccess;
    const cudaMemcpyKind kind = where == SIPF_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (x) {
        e = launch_export_positions_inplace(c, o);
        const float* arr[3] = {c->sx[o], c->sy[o], c->sz[o]};
        for (int d = 0; d < 3 && e == cudaSuccess; ++d)
            e = cudaMemcpyAsync(x + d * N, arr[d], N * sizeof(float), kind, c->stream);
    }
    if (e == cudaSuccess && mass) {
        e = launch_export_mass(c, o, c->dl[o], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(mass, c->dl[o], N * sizeof(double), kind, c->stream);
    }
    if (e == cudaSuccess && id)
        e = cudaMemcpyAsync(id, c->id[o], N * sizeof(uint32_t), kind, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "sipf_particles");
    return check_status(c);
}

int sipf_cell_start(sipf_ctx* c, int32_t* cell_start, int where) {
    if (!c || !cell_start) return SIPF_EINVAL;
    if (where != SIPF_HOST && where != SIPF_DEVICE) return fail(c, SIPF_EINVAL, "bad where");
    if (!c->state_set) return fail(c, SIPF_EINVAL, "sipf_set_state has not been called");
    const size_t H3 = static_cast<size_t>(c->H) * c->H * c->H;
    int r = compact_current(c);
    if (r != SIPF_OK) return r;
    SIPF_CUDA(c, launch_cell_histogram(c, c->cur ^ 1, c->count, c->scan_tmp, c->cell_start));
    r = copy_out(c, cell_start, c->cell_start, (H3 + 1) * sizeof(int32_t), where);
    if (r != SIPF_OK) return r;
    return check_status(c);
}

int sipf_set_tuning(sipf_ctx* c, const sipf_tuning* t) {
    if (!c || !t) return SIPF_EINVAL;
    if (!tuning_valid(*t)) return fail(c, SIPF_EINVAL, "tuning out of range");
    // captured step graphs bake in the kernels and launch shapes
    cudaStreamSynchronize(c->stream);
    for (const auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
    apply_tuning(c, *t);
    c->step_blocks = step_grid(c);
    return SIPF_OK;
}

int sipf_get_tuning(const sipf_ctx* c, sipf_tuning* t) {
    if (!c || !t) return SIPF_EINVAL;
    t->radix_plan = c->radix_plan;
    t->step_blocks_per_sm = c->step_bps;
    t->bucket_slack_div = c->slack_div;
    t->bucket_slack_add = c->slack_add;
    return SIPF_OK;
}

int sipf_tuning_load(const char* path) {
    std::vector<TuneEntry> t;
    if (path) {
        const int r = parse_tuning_file(path, &t);
        if (r != SIPF_OK) return r;
    }
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune = t;
    g_tune_loaded = true;
    return SIPF_OK;
}

int sipf_tuning_lookup(int32_t H, int64_t N, sipf_tuning* out) {
    if (!out) return SIPF_EINVAL;
    return lookup_tuning(H, N, out) ? 1 : 0;
}

int sipf_canonical_order(sipf_ctx* c, int32_t* cell_start, uint32_t* ids, int where) {
    if (!c || (!cell_start && !ids)) return SIPF_EINVAL;
    if (where != SIPF_HOST && where != SIPF_DEVICE) return fail(c, SIPF_EINVAL, "bad where");
    if (!c->state_set) return fail(c, SIPF_EINVAL, "sipf_set_state has not been called");
    const size_t H3 = static_cast<size_t>(c->H) * c->H * c->H;
    int r = compact_current(c);
    if (r != SIPF_OK) return r;
    const int o = c->cur ^ 1;
    SIPF_CUDA(c, launch_canonical_order(c, o));
    if (cell_start) r = copy_out(c, cell_start, c->cell_start, (H3 + 1) * sizeof(int32_t), where);
    if (r == SIPF_OK && ids)
        r = copy_out(c, ids, c->id[o], static_cast<size_t>(c->N) * sizeof(uint32_t), where);
    if (r != SIPF_OK) return r;
    return check_status(c);
}

int sipf_diagnostics(sipf_ctx* c, sipf_diag* out) {
    if (!c || !out) return SIPF_EINVAL;
    if (!c->state_set) return fail(c, SIPF_EINVAL, "sipf_set_state has not been called");
    int r = compact_current(c);
    if (r == SIPF_OK) r = deposit_current(c);
    if (r != SIPF_OK) return r;
    SIPF_CUDA(c, launch_diagnostics(c, c->cur ^ 1, acc_to_u_d(c)));
    const size_t H3 = static_cast<size_t>(c->H) * c->H * c->H;
    SIPF_CUDA(c, cudaMemsetAsync(c->acc, 0, H3 * sizeof(long long), c->stream));
    double h[8];
    SIPF_CUDA(c, cudaMemcpyAsync(h, c->diag_out, 7 * sizeof(double), cudaMemcpyDeviceToHost,
                                 c->stream));
    SIPF_CUDA(c, cudaStreamSynchronize(c->stream));
    out->mass_particles = h[0];
    out->mass_grid = h[1] * c->h * c->h * c->h;
    out->min_u = h[2];
    out->min_v = h[3];
    out->min_m = h[4];
    out->min_w = h[5];
    out->nonfinite = static_cast<int64_t>(h[6]);
    out->step = c->step;
    out->time = c->time;
    return check_status(c);
}

int sipf_sync(sipf_ctx* c) {
    if (!c) return SIPF_EINVAL;
    return check_status(c);
}

void sipf_destroy(sipf_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (cudaEvent_t e : c->prof_events) cudaEventDestroy(e);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    for (const auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    free_all(c);
    delete c;
}

int sipf_save(sipf_ctx* c, const char* path) {
    if (!c) return SIPF_EINVAL;
    if (!path) return fail(c, SIPF_EINVAL, "NULL path");
    if (!c->state_set) return fail(c, SIPF_EINVAL, "sipf_set_state has not been called");
    const size_t N = static_cast<size_t>(c->N);
    const size_t H3 = static_cast<size_t>(c->H) * c->H * c->H;
    int r = compact_current(c);
    if (r != SIPF_OK) return r;
    const int o = c->cur ^ 1;
    const CkptArray arrays[] = {
        {c->sx[o], N * sizeof(float)}, {c->sy[o], N * sizeof(float)},
        {c->sz[o], N * sizeof(float)}, {c->dl[o], N * sizeof(double)},
        {c->id[o], N * sizeof(uint32_t)}, {c->v, H3 * sizeof(float)},
        {c->m, H3 * sizeof(float)}, {c->w, H3 * sizeof(float)}, {c->G, 4 * H3 * sizeof(float)}};
    size_t total = 0;
    for (const CkptArray& a : arrays) total += a.bytes;
    std::vector<unsigned char> payload;
    try {
        payload.resize(total);
    } catch (...) {
        return fail(c, SIPF_ENOMEM, "sipf_save: host buffer");
    }
    size_t off = 0;
    for (const CkptArray& a : arrays) {
        SIPF_CUDA(c, cudaMemcpyAsync(payload.data() + off, a.dev, a.bytes, cudaMemcpyDeviceToHost,
                                     c->stream));
        off += a.bytes;
    }
    float voff = 0.f;
    SIPF_CUDA(c, cudaMemcpyAsync(&voff, c->voff, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    SIPF_CUDA(c, cudaStreamSynchronize(c->stream));
    r = check_status(c);
    if (r != SIPF_OK) return r;
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, kCkptMagic, 8);
    hd.version = kCkptVersion;
    hd.header_bytes = sizeof(CkptHeader);
    hd.H = c->H;
    hd.L = c->L;
    for (int k = 0; k < 3; ++k) hd.origin[k] = c->origin[k];
    hd.N = c->N;
    hd.params = c->p;
    hd.step = c->step;
    hd.time = c->time;
    hd.logref = c->logref;
    hd.maxrel = c->maxrel;
    hd.voff = voff;
    hd.payload_bytes = total;
    hd.payload_hash = ckpt_hash(0xCBF29CE484222325ull, payload.data(), total);
    FILE* f = fopen(path, "wb");
    if (!f) return fail(c, SIPF_EINVAL, std::string("sipf_save: cannot open ") + path);
    const bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 &&
                    fwrite(payload.data(), 1, total, f) == total;
    const bool closed = fclose(f) == 0;
    if (!ok || !closed) return fail(c, SIPF_EINVAL, std::string("sipf_save: write failed: ") + path);
    return SIPF_OK;
}

int sipf_load(const char* path, void* stream, sipf_ctx** out) {
    if (!path || !out) return SIPF_EINVAL;
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return SIPF_EINVAL;
    CkptHeader hd;
    if (fread(&hd, sizeof(hd), 1, f) != 1 || memcmp(hd.magic, kCkptMagic, 8) != 0 ||
        hd.version != kCkptVersion || hd.header_bytes != sizeof(CkptHeader) ||
        !supported_H(hd.H) || hd.N < 1 || hd.N >= (int64_t{1} << 31)) {
        fclose(f);
        return SIPF_EINVAL;
    }
    const size_t N = static_cast<size_t>(hd.N);
    const size_t H3 = static_cast<size_t>(hd.H) * hd.H * hd.H;
    const size_t total = N * (3 * sizeof(float) + sizeof(double) + sizeof(uint32_t)) +
                         H3 * 7 * sizeof(float);
    if (hd.payload_bytes != total) {
        fclose(f);
        return SIPF_EINVAL;
    }
    std::vector<unsigned char> payload;
    try {
        payload.resize(total);
    } catch (...) {
        fclose(f);
        return SIPF_ENOMEM;
    }
    const bool got = fread(payload.data(), 1, total, f) == total;
    fclose(f);
    if (!got || ckpt_hash(0xCBF29CE484222325ull, payload.data(), total) != hd.payload_hash)
        return SIPF_EINVAL;
    sipf_grid g;
    g.H = hd.H;
    g.L = hd.L;
    for (int k = 0; k < 3; ++k) g.origin[k] = hd.origin[k];
    sipf_ctx* c = nullptr;
    int r = sipf_create(&g, hd.N, &hd.params, stream, &c);
    if (r != SIPF_OK) return r;
    // particles unbinned into buffer 1, fields and the gather array as saved
    const CkptArray arrays[] = {
        {c->sx[1], N * sizeof(float)}, {c->sy[1], N * sizeof(float)},
        {c->sz[1], N * sizeof(float)}, {c->dl[1], N * sizeof(double)},
        {c->id[1], N * sizeof(uint32_t)}, {c->v, H3 * sizeof(float)},
        {c->m, H3 * sizeof(float)}, {c->w, H3 * sizeof(float)}, {c->G, 4 * H3 * sizeof(float)}};
    size_t off = 0;
    cudaError_t e = cudaSuccess;
    for (const CkptArray& a : arrays) {
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(a.dev, payload.data() + off, a.bytes, cudaMemcpyHostToDevice,
                                c->stream);
        off += a.bytes;
    }
    c->voff_host = hd.voff;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->voff, &c->voff_host, sizeof(float), cudaMemcpyHostToDevice,
                            c->stream);
    c->step = hd.step;
    c->time = hd.time;
    c->logref = hd.logref;
    c->maxrel = hd.maxrel;
    set_mass_reference(c);
    if (e == cudaSuccess) {
        r = bin_initial(c);
        if (r == SIPF_OK) r = write_scalars(c);
        if (r == SIPF_OK) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess || r != SIPF_OK || check_status(c) != SIPF_OK) {
        sipf_destroy(c);
        return e != cudaSuccess ? SIPF_ECUDA : (r != SIPF_OK ? r : SIPF_EINTERNAL);
    }
    c->state_set = true;
    *out = c;
    return SIPF_OK;
}

int sipf_resample(sipf_ctx* c, double ratio, int32_t* resampled) {
    if (!c) return SIPF_EINVAL;
    if (resampled) *resampled = 0;
    if (!c->state_set) return fail(c, SIPF_EINVAL, "sipf_set_state has not been called");
    if (!isfinite(ratio)) return fail(c, SIPF_EINVAL, "ratio must be finite");
    // compacted particles in the free buffer; the binned one is then free too
    int r = compact_current(c);
    if (r != SIPF_OK) return r;
    const int src = c->cur ^ 1, dst = c->cur;
    int done = 0;
    std::string why;
    r = resample_device(c, src, dst, ratio, &done, &why);
    if (r != SIPF_OK) return fail(c, r, "sipf_resample: " + why);
    if (done) {
        r = bin_from(c, dst);
        if (r == SIPF_OK) r = write_scalars(c);
        if (r != SIPF_OK) return r;
        SIPF_CUDA(c, cudaStreamSynchronize(c->stream));
        r = check_status(c);
        if (r != SIPF_OK) return r;
    }
    if (resampled) *resampled = done;
    return SIPF_OK;
}

int64_t sipf_context_bytes(const sipf_grid* grid, int64_t N, const sipf_params* params) {
    std::string why;
    if (!grid || !params || N < 1 || N >= (int64_t{1} << 31) || !supported_H(grid->H) ||
        check_params(params, &why) != SIPF_OK)
        return SIPF_EINVAL;
    if (ctx_sizes(grid->H, N).buf_slots >= (int64_t{1} << 31)) return SIPF_EINVAL;
    const bool filter = params->H0 > 0.0 && params->H0 < grid->H;
    return static_cast<int64_t>(ctx_device_bytes(grid->H, N, filter, params->sigma > 0.0));
}

int64_t sipf_device_bytes(const sipf_ctx* c) {
    return c ? static_cast<int64_t>(c->dev_bytes) : SIPF_EINVAL;
}

int sipf_describe(const sipf_ctx* c, sipf_grid* grid, int64_t* N, sipf_params* params,
                  int64_t* step, double* time) {
    if (!c) return SIPF_EINVAL;
    if (grid) {
        grid->H = c->H;
        grid->L = c->L;
        for (int k = 0; k < 3; ++k) grid->origin[k] = c->origin[k];
    }
    if (N) *N = c->N;
    if (params) *params = c->p;
    if (step) *step = c->step;
    if (time) *time = c->time;
    return SIPF_OK;
}

// ---------------------------------------------------------------- ensembles
}  // extern "C"

struct sipf_ensemble {
    std::vector<sipf_ctx*> members;
    std::vector<cudaStream_t> streams;   // one per member, owned here
    int mode = SIPF_ENSEMBLE_BATCHED;
    int last_path = -1;
    // batched steps: the ensemble's own streams and events, and the captured
    // two-step graphs, each with the run table its kernels read
    cudaStream_t main = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_done = nullptr;
    std::vector<cudaEvent_t> ev_member;
    struct BatchGraph {
        std::vector<double> dt;
        int parity;
        cudaGraphExec_t exec;
        sipf::RunDesc* d_runs;
    };
    std::vector<BatchGraph> graphs;
    std::string last_error;
};

namespace {
void ensemble_free(sipf_ensemble* e) {
    if (e->main) cudaStreamSynchronize(e->main);
    if (e->side) cudaStreamSynchronize(e->side);
    for (auto& g : e->graphs) {
        cudaGraphExecDestroy(g.exec);
        cudaFree(g.d_runs);
    }
    for (sipf_ctx* c : e->members)
        if (c) sipf_destroy(c);
    for (cudaStream_t s : e->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t ev : e->ev_member) cudaEventDestroy(ev);
    for (cudaEvent_t ev : {e->ev_fork, e->ev_join, e->ev_done})
        if (ev) cudaEventDestroy(ev);
    if (e->main) cudaStreamDestroy(e->main);
    if (e->side) cudaStreamDestroy(e->side);
    delete e;
}
}  // namespace

extern "C" {

}  // extern "C"

namespace {

// The batched step applies when every member uses the trilinear assignment
// without the filter or the K_sigma source, has a fused-pass grid (H <= 128),
// a stream of its own and no tracing, and all members read the same buffer
// parity.
bool batchable(const sipf_ensemble* e) {
    if (e->members.empty() || e->members.size() > static_cast<size_t>(kMaxRuns)) return false;
    const int parity = e->members[0]->cur;
    for (const sipf_ctx* c : e->members) {
        const bool filter = c->p.H0 > 0.0 && c->p.H0 < c->H;
        if (c->p.p2g_order != 2 || filter || c->us || c->H > 128 || !c->stream || c->prof_on ||
            c->cur != parity)
            return false;
    }
    return true;
}

// One batched step of every member from buffer `parity`: the particle step
// of all runs in one persistent launch, the plans of all runs in one launch
// on the second stream, and each fused spectral pass once per grid size
// (runs of one size batched into one launch).
int enqueue_batched_step(sipf_ensemble* e, const double* dt, const RunDesc* d_runs, int parity) {
    const int n = static_cast<int>(e->members.size());
    auto cuda = [e](cudaError_t err, const char* where) {
        if (err == cudaSuccess) return SIPF_OK;
        cudaGetLastError();
        e->last_error = std::string(where) + ": " + cudaGetErrorString(err);
        return SIPF_ECUDA;
    };
    int r = cuda(launch_step_multi(d_runs, n, parity, e->main), "batched particle step");
    if (r == SIPF_OK) r = cuda(cudaEventRecord(e->ev_fork, e->main), "cudaEventRecord");
    if (r == SIPF_OK) r = cuda(cudaStreamWaitEvent(e->side, e->ev_fork, 0), "cudaStreamWaitEvent");
    if (r == SIPF_OK) r = cuda(launch_plan_multi(d_runs, n, parity, e->side), "batched plan");
    if (r == SIPF_OK) r = cuda(cudaEventRecord(e->ev_join, e->side), "cudaEventRecord");
    // runs grouped by (grid size, radix plan), in member order within a
    // group, so that every member runs the passes of its own plan
    std::vector<std::pair<int, int>> groups;
    for (const sipf_ctx* c : e->members) {
        const std::pair<int, int> g(c->H, c->radix_plan);
        if (std::find(groups.begin(), groups.end(), g) == groups.end()) groups.push_back(g);
    }
    std::sort(groups.begin(), groups.end());
    const int device = e->members[0]->device;
    for (const auto& g : groups) {
        const int H = g.first, plan = g.second;
        std::vector<SpecRun> runs;
        for (int i = 0; i < n; ++i)
            if (e->members[i]->H == H && e->members[i]->radix_plan == plan)
                runs.push_back(spec_run(e->members[i], spectral_args(e->members[i], dt[i], 1)));
        for (size_t b0 = 0; b0 < runs.size() && r == SIPF_OK; b0 += kMaxBatch) {
            const int nb = static_cast<int>(std::min<size_t>(kMaxBatch, runs.size() - b0));
            for (int pass = 0; pass < 3 && r == SIPF_OK; ++pass)
                r = cuda(launch_spectral_batch(H, runs.data() + b0, nb, pass, plan, device,
                                               e->main),
                         "batched spectral pass");
        }
    }
    if (r == SIPF_OK) r = cuda(cudaStreamWaitEvent(e->main, e->ev_join, 0), "cudaStreamWaitEvent");
    if (r != SIPF_OK) return r;
    for (int i = 0; i < n; ++i) advance_host(e->members[i], dt[i]);
    return SIPF_OK;
}

// The two-step graph of the current parity and dt vector (captured on the
// first call), with its run table.
int batched_graph(sipf_ensemble* e, const double* dt, sipf_ensemble::BatchGraph** out) {
    *out = nullptr;
    const size_t n = e->members.size();
    const int parity = e->members[0]->cur;
    std::vector<double> dts(dt, dt + n);
    for (auto& g : e->graphs)
        if (g.parity == parity && g.dt == dts) {
            *out = &g;
            return SIPF_OK;
        }
    std::vector<RunDesc> host(n);
    for (size_t i = 0; i < n; ++i) host[i] = run_desc(e->members[i], dt[i]);
    RunDesc* d_runs = nullptr;
    if (cudaMalloc(&d_runs, n * sizeof(RunDesc)) != cudaSuccess ||
        cudaMemcpy(d_runs, host.data(), n * sizeof(RunDesc), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        if (d_runs) cudaFree(d_runs);
        e->last_error = "run table of the batched step";
        return SIPF_ENOMEM;
    }
    std::vector<int> cur0(n);
    std::vector<int64_t> step0(n);
    std::vector<double> time0(n);
    for (size_t i = 0; i < n; ++i) {
        cur0[i] = e->members[i]->cur;
        step0[i] = e->members[i]->step;
        time0[i] = e->members[i]->time;
    }
    if (cudaStreamBeginCapture(e->main, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_runs);
        e->last_error = "stream capture of the batched step";
        return SIPF_ECUDA;
    }
    int r = enqueue_batched_step(e, dt, d_runs, parity);
    if (r == SIPF_OK) r = enqueue_batched_step(e, dt, d_runs, parity ^ 1);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(e->main, &graph);
    for (size_t i = 0; i < n; ++i) {
        e->members[i]->cur = cur0[i];
        e->members[i]->step = step0[i];
        e->members[i]->time = time0[i];
    }
    cudaGraphExec_t exec = nullptr;
    const bool ok = r == SIPF_OK && ce == cudaSuccess && graph &&
                    cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        cudaFree(d_runs);
        if (r == SIPF_OK) e->last_error = "instantiating the batched step graph";
        return r == SIPF_OK ? SIPF_ECUDA : r;
    }
    if (e->graphs.size() >= 4) {
        cudaGraphExecDestroy(e->graphs.front().exec);
        cudaFree(e->graphs.front().d_runs);
        e->graphs.erase(e->graphs.begin());
    }
    e->graphs.push_back({dts, parity, exec, d_runs});
    *out = &e->graphs.back();
    return SIPF_OK;
}

// k batched steps: the members' streams are ordered before and after the
// ensemble's own stream, pairs of steps replay the captured graph, an odd
// last step is enqueued launch by launch with the graph's run table.
int batched_steps(sipf_ensemble* e, const double* dt, int64_t k) {
    const size_t n = e->members.size();
    for (size_t i = 0; i < n; ++i) {
        if (cudaEventRecord(e->ev_member[i], e->members[i]->stream) != cudaSuccess ||
            cudaStreamWaitEvent(e->main, e->ev_member[i], 0) != cudaSuccess) {
            cudaGetLastError();
            e->last_error = "ordering the member streams";
            return SIPF_ECUDA;
        }
    }
    int r = SIPF_OK;
    for (int64_t done = 0; done < k && r == SIPF_OK;) {
        sipf_ensemble::BatchGraph* g = nullptr;
        r = batched_graph(e, dt, &g);
        if (r != SIPF_OK) break;
        if (k - done >= 2) {
            if (cudaGraphLaunch(g->exec, e->main) != cudaSuccess) {
                cudaGetLastError();
                e->last_error = "cudaGraphLaunch";
                r = SIPF_ECUDA;
                break;
            }
            for (size_t i = 0; i < n; ++i) {
                advance_host(e->members[i], dt[i]);
                advance_host(e->members[i], dt[i]);
            }
            done += 2;
        } else {
            r = enqueue_batched_step(e, dt, g->d_runs, e->members[0]->cur);
            done += 1;
        }
    }
    // later calls on a member (fields, diagnostics, ...) follow the batched work
    if (cudaEventRecord(e->ev_done, e->main) != cudaSuccess) r = SIPF_ECUDA;
    for (size_t i = 0; i < n; ++i)
        if (cudaStreamWaitEvent(e->members[i]->stream, e->ev_done, 0) != cudaSuccess) r = SIPF_ECUDA;
    if (r == SIPF_ECUDA) cudaGetLastError();
    return r;
}

}  // namespace

extern "C" {

int sipf_ensemble_create(int32_t count, const sipf_grid* grids, const int64_t* N,
                         const sipf_params* params, sipf_ensemble** out) {
    if (!out) return SIPF_EINVAL;
    *out = nullptr;
    if (count < 1 || !grids || !N || !params) return SIPF_EINVAL;
    sipf_ensemble* e = new (std::nothrow) sipf_ensemble();
    if (!e) return SIPF_ENOMEM;
    for (int32_t i = 0; i < count; ++i) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            ensemble_free(e);
            return SIPF_ECUDA;
        }
        e->streams.push_back(s);
        sipf_ctx* c = nullptr;
        const int r = sipf_create(&grids[i], N[i], &params[i], s, &c);
        if (r != SIPF_OK) {
            ensemble_free(e);
            return r;
        }
        e->members.push_back(c);
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            ensemble_free(e);
            return SIPF_ECUDA;
        }
        e->ev_member.push_back(ev);
    }
    if (cudaStreamCreateWithFlags(&e->main, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&e->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->ev_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ensemble_free(e);
        return SIPF_ECUDA;
    }
    *out = e;
    return SIPF_OK;
}

sipf_ctx* sipf_ensemble_member(sipf_ensemble* e, int32_t i) {
    if (!e || i < 0 || i >= static_cast<int32_t>(e->members.size())) return nullptr;
    return e->members[i];
}

int sipf_ensemble_set_mode(sipf_ensemble* e, int mode) {
    if (!e || (mode != SIPF_ENSEMBLE_BATCHED && mode != SIPF_ENSEMBLE_STREAMS)) return SIPF_EINVAL;
    e->mode = mode;
    return SIPF_OK;
}

int sipf_ensemble_last_path(const sipf_ensemble* e) { return e ? e->last_path : SIPF_EINVAL; }

int sipf_ensemble_step(sipf_ensemble* e, const double* dt, int64_t k) {
    if (!e || !dt || k < 0) return SIPF_EINVAL;
    for (size_t i = 0; i < e->members.size(); ++i) {
        sipf_ctx* c = e->members[i];
        if (!c->state_set) {
            e->last_error = "member " + std::to_string(i) + ": sipf_set_state has not been called";
            return SIPF_EINVAL;
        }
        if (!(isfinite(dt[i]) && dt[i] > 0.0 && dt[i] <= 0.5)) {
            e->last_error = "member " + std::to_string(i) + ": dt must satisfy 0 < dt <= 0.5";
            return SIPF_EINVAL;
        }
    }
    if (k == 0) return SIPF_OK;
    if (e->mode == SIPF_ENSEMBLE_BATCHED && batchable(e)) {
        e->last_path = SIPF_ENSEMBLE_BATCHED;
        return batched_steps(e, dt, k);
    }
    e->last_path = SIPF_ENSEMBLE_STREAMS;
    // every member's work goes to its own stream, so the kernels of different
    // members run concurrently; pairs of steps replay each member's captured
    // two-step graph, interleaved member after member
    const size_t M = e->members.size();
    std::vector<cudaGraphExec_t> exec(M, nullptr);
    for (size_t i = 0; i < M && k >= 2; ++i) {
        sipf_ctx* c = e->members[i];
        if (c->prof_on) continue;
        const int r = step_pair_graph(c, dt[i], &exec[i]);
        if (r != SIPF_OK) {
            e->last_error = "member " + std::to_string(i) + ": " + c->last_error;
            return r;
        }
    }
    int64_t n = 0;
    for (; n + 2 <= k; n += 2) {
        for (size_t i = 0; i < M; ++i) {
            sipf_ctx* c = e->members[i];
            int r = SIPF_OK;
            if (exec[i]) {
                const cudaError_t ce = cudaGraphLaunch(exec[i], c->stream);
                if (ce == cudaSuccess) {
                    advance_host(c, dt[i]);
                    advance_host(c, dt[i]);
                } else {
                    r = cuda_fail(c, ce, "cudaGraphLaunch");
                }
            } else {
                r = enqueue_step(c, dt[i]);
                if (r == SIPF_OK) r = enqueue_step(c, dt[i]);
            }
            if (r != SIPF_OK) {
                e->last_error = "member " + std::to_string(i) + ": " + c->last_error;
                return r;
            }
        }
    }
    for (; n < k; ++n) {
        for (size_t i = 0; i < M; ++i) {
            const int r = enqueue_step(e->members[i], dt[i]);
            if (r != SIPF_OK) {
                e->last_error = "member " + std::to_string(i) + ": " + e->members[i]->last_error;
                return r;
            }
        }
    }
    return SIPF_OK;
}

int sipf_ensemble_sync(sipf_ensemble* e) {
    if (!e) return SIPF_EINVAL;
    int first = SIPF_OK;
    for (size_t i = 0; i < e->members.size(); ++i) {
        const int r = sipf_sync(e->members[i]);
        if (r != SIPF_OK && first == SIPF_OK) {
            first = r;
            e->last_error = "member " + std::to_string(i) + ": " + e->members[i]->last_error;
        }
    }
    return first;
}

const char* sipf_ensemble_last_error(const sipf_ensemble* e) {
    return e ? e->last_error.c_str() : "";
}

void sipf_ensemble_destroy(sipf_ensemble* e) {
    if (e) ensemble_free(e);
}

int sipf_profile(sipf_ctx* c, int enable) {
    if (!c) return SIPF_EINVAL;
    if (enable && !c->prof_on) c->prof_steps = 0;
    c->prof_on = enable != 0;
    return SIPF_OK;
}

int sipf_profile_read(sipf_ctx* c, double* ms, int64_t* launches, int n) {
    if (!c || !ms || !launches || n < 1) return SIPF_EINVAL;
    SIPF_CUDA(c, cudaStreamSynchronize(c->stream));
    static const int per_step[kProfGroups] = {1, 1, 1, 1};
    for (int k = 0; k < n; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    for (int64_t s = 0; s < c->prof_steps; ++s) {
        for (int k = 0; k < kProfGroups && k < n; ++k) {
            const size_t i = static_cast<size_t>(s) * (kProfGroups + 1) + k;
            float t = 0.f;
            SIPF_CUDA(c, cudaEventElapsedTime(&t, c->prof_events[i], c->prof_events[i + 1]));
            ms[k] += t;
            launches[k] += per_step[k];
        }
    }
    return SIPF_OK;
}

const char* sipf_profile_name(int k) {
    static const char* names[kProfGroups] = {"particle_step", "forward_xy", "z_multiply",
                                             "inverse_xy"};
    return (k >= 0 && k < kProfGroups) ? names[k] : "";
}

int sipf_brownian_normals(const uint32_t* ids, int64_t N, uint32_t n, uint64_t seed, float* z,
                          uint32_t* bits, void* stream) {
    if (!ids || !z || N < 1 || N >= (int64_t{1} << 31)) return SIPF_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (launch_normals(ids, N, n, seed, z, bits, s) != cudaSuccess) return SIPF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SIPF_ECUDA;
    return SIPF_OK;
}

}  // extern "C"
