// C ABI of liblbm.so (declarations and contracts: include/lbm.h).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/lbm.h"
#include "adjoint_kernels.cuh"

namespace lbm {
LBM_INSTANTIATE(extern, 27)
LBM_INSTANTIATE(extern, 15)
LBM_INSTANTIATE_ADJOINT(extern, 27, float)
LBM_INSTANTIATE_ADJOINT(extern, 15, float)
LBM_INSTANTIATE_ADJOINT(extern, 27, __half)
LBM_INSTANTIATE_ADJOINT(extern, 15, __half)
LBM_INSTANTIATE_ADJOINT(extern, 27, __nv_bfloat16)
LBM_INSTANTIATE_ADJOINT(extern, 15, __nv_bfloat16)
}  // namespace lbm

// A captured run of steps (a CUDA graph), valid for the launch arguments,
// buffers and starting parity in its key.
struct GraphKey {
    int Q, storage, nx, ny, nz, px, layout, cur, steps, has_force;
    unsigned bc;
    float w[27], F[3];
    const float *Ffield;
    const void *buf0, *buf1;
};
struct StepGraph {
    GraphKey key;
    cudaGraphExec_t exec;
    unsigned long long used;  // for least-recently-used replacement
};

struct lbm_ctx {
    int Q;
    lbm_storage storage;
    lbm::Grid g;
    float w[27];
    float F[3];
    void *buf[2];
    int cur;  // buffer holding the current state
    const float *Ffield;
    bool bound;
    bool state_set;
    bool inplace;  // single-buffer (AA) streaming; g.layout tracks the state's layout
    bool sr32;     // stochastically rounded FP32 update (LBM_F32_SR)
    int device;
    int graph_steps;          // steps per captured graph; 0: launch each step
    cudaStream_t cap_stream;  // private stream the graphs are captured on
    StepGraph graphs[2];      // one per starting parity, typically
    unsigned long long graph_clock;
    double *red_scratch;  // partial sums + 4 totals
    int red_blocks;
    const char *cuda_error;
};

namespace {

constexpr int kDefaultGraphSteps = 32;

size_t elem_bytes(lbm_storage st) { return st == LBM_STORE_F32 ? 4 : 2; }

lbm::StepArgs step_args(const lbm_ctx *c) {
    lbm::StepArgs a;
    a.g = c->g;
    for (int b = 0; b < 27; ++b) a.w[b] = c->w[b];
    for (int i = 0; i < 3; ++i) a.F[i] = c->F[i];
    a.Ffield = c->Ffield;
    a.has_force = (c->Ffield || c->F[0] != 0.0f || c->F[1] != 0.0f || c->F[2] != 0.0f) ? 1 : 0;
    a.sr32 = c->sr32 ? 1 : 0;
    return a;
}

bool valid_rates(int Q, const double *omega) {
    if (!omega) return false;
    for (int b = 4; b < Q; ++b)
        if (!(omega[b] > 0.0 && omega[b] < 2.0)) return false;
    return true;
}

lbm_status cuda_fail(const lbm_ctx *c, cudaError_t e) {
    const_cast<lbm_ctx *>(c)->cuda_error = cudaGetErrorString(e);
    return LBM_ECUDA;
}

// Every field set one by one on a zeroed key, so keys compare bytewise.
GraphKey graph_key(const lbm_ctx *c, int steps) {
    GraphKey k;
    std::memset(&k, 0, sizeof(k));
    k.Q = c->Q;
    k.storage = int(c->storage);
    k.nx = c->g.nx;
    k.ny = c->g.ny;
    k.nz = c->g.nz;
    k.px = c->g.px;
    k.layout = c->g.layout;
    k.cur = c->cur;
    k.steps = steps;
    k.bc = c->g.bc;
    for (int b = 0; b < 27; ++b) k.w[b] = c->w[b];
    for (int i = 0; i < 3; ++i) k.F[i] = c->F[i];
    k.Ffield = c->Ffield;
    k.has_force = step_args(c).has_force;
    k.buf0 = c->buf[0];
    k.buf1 = c->buf[1];
    return k;
}

void drop_graphs(lbm_ctx *c) {
    for (StepGraph &g : c->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        g.used = 0;
    }
}

// Dispatch on (Q, storage) to a templated launcher F<Q, T>.
template <template <int, typename> class Fn, typename... Args>
cudaError_t dispatch(const lbm_ctx *c, Args &&...args) {
    switch (c->Q * 4 + int(c->storage)) {
        case 27 * 4 + LBM_STORE_F32: return Fn<27, float>::run(args...);
        case 27 * 4 + LBM_STORE_F16: return Fn<27, __half>::run(args...);
        case 27 * 4 + LBM_STORE_BF16: return Fn<27, __nv_bfloat16>::run(args...);
        case 15 * 4 + LBM_STORE_F32: return Fn<15, float>::run(args...);
        case 15 * 4 + LBM_STORE_F16: return Fn<15, __half>::run(args...);
        case 15 * 4 + LBM_STORE_BF16: return Fn<15, __nv_bfloat16>::run(args...);
        default: return cudaErrorInvalidValue;
    }
}

template <int Q, typename T>
struct AdjointFn {
    static cudaError_t run(const void *f, const float *ln, float *lo, float *gF,
                           const lbm::StepArgs &a, cudaStream_t s) {
        return lbm::launch_adjoint<Q, T>(f, ln, lo, gF, a, s);
    }
};
template <int Q, typename T>
struct SeedFn {
    static cudaError_t run(const void *f, float *lo, float *gF, const lbm::StepArgs &a,
                           cudaStream_t s) {
        return lbm::launch_energy_seed<Q, T>(f, lo, gF, a, s);
    }
};
template <int Q, typename T>
struct MacroSeedFn {
    static cudaError_t run(const void *f, const float *g_rho, const float *g_u, float *lo,
                           float *gF, const lbm::StepArgs &a, cudaStream_t s) {
        return lbm::launch_macro_seed<Q, T>(f, g_rho, g_u, lo, gF, a, s);
    }
};
template <int Q, typename T>
struct EnergyFn {
    static cudaError_t run(const void *f, const lbm::StepArgs &a, double *part, int blocks,
                           cudaStream_t s) {
        return lbm::launch_energy<Q, T>(f, a, part, blocks, s);
    }
};

template <int Q, typename T>
struct StepFn {
    static cudaError_t run(const void *fin, void *fout, const lbm::StepArgs &a, cudaStream_t s) {
        return lbm::launch_step<Q, T>(fin, fout, a, s);
    }
};
template <int Q, typename T>
struct StepAAFn {
    static cudaError_t run(void *buf, const lbm::StepArgs &a, bool even, cudaStream_t s) {
        return lbm::launch_step_aa<Q, T>(buf, a, even, s);
    }
};
template <int Q, typename T>
struct InitFn {
    static cudaError_t run(void *buf, const lbm::StepArgs &a, const double *rho, const double *u,
                           cudaStream_t s) {
        return lbm::launch_init<Q, T>(buf, a, rho, u, s);
    }
};
template <int Q, typename T>
struct SetFn {
    static cudaError_t run(void *buf, const lbm::Grid &g, const double *f, cudaStream_t s) {
        return lbm::launch_set_state<Q, T>(buf, g, f, s);
    }
};
template <int Q, typename T>
struct GetFn {
    static cudaError_t run(const void *buf, const lbm::Grid &g, double *f, cudaStream_t s) {
        return lbm::launch_get_state<Q, T>(buf, g, f, s);
    }
};
template <int Q, typename T>
struct MacroFn {
    static cudaError_t run(const void *buf, const lbm::StepArgs &a, float *rho, float *u,
                           cudaStream_t s) {
        return lbm::launch_macro<Q, T>(buf, a, rho, u, s);
    }
};
template <int Q, typename T>
struct ConsFn {
    static cudaError_t run(const void *buf, const lbm::StepArgs &a, double *part, int blocks,
                           cudaStream_t s) {
        return lbm::launch_conservation<Q, T>(buf, a, part, blocks, s);
    }
};

}  // namespace

extern "C" {

lbm_status lbm_create(lbm_lattice lattice, int nx, int ny, int nz, const double *omega,
                      const double *force, unsigned bc_flags, lbm_storage storage,
                      lbm_ctx **out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    const int Q = int(lattice);
    if (Q != 27 && Q != 15) return LBM_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1) return LBM_EINVAL;
    if (ny > 65535 || nz > 65535) return LBM_EINVAL;  // launch grid limits (y, z)
    if (bc_flags & ~(LBM_WALL_Y | LBM_WALL_Z | LBM_INPLACE | LBM_F32_SR)) return LBM_EINVAL;
    const bool inplace = (bc_flags & LBM_INPLACE) != 0;
    const bool sr32 = (bc_flags & LBM_F32_SR) != 0;
    if (sr32 && (inplace || storage != LBM_STORE_F32)) return LBM_EINVAL;
    if (inplace && (nx % 2) != 0) return LBM_EINVAL;  // the in-place kernels take cell pairs
    if (storage != LBM_STORE_F32 && storage != LBM_STORE_F16 && storage != LBM_STORE_BF16)
        return LBM_EINVAL;
    if (!valid_rates(Q, omega)) return LBM_EINVAL;
    const long long px = ((long long)nx + 31) / 32 * 32;
    const long long cells = (long long)nx * ny * nz;
    // population planes are addressed with 32-bit element offsets
    if (px * ny * nz >= (1LL << 31) || cells >= (1LL << 31)) return LBM_EINVAL;
    if (force)
        for (int i = 0; i < 3; ++i)
            if (!std::isfinite(force[i])) return LBM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ENOMEM;
    c->Q = Q;
    c->storage = storage;
    c->g.nx = nx;
    c->g.ny = ny;
    c->g.nz = nz;
    c->g.px = int(px);
    c->g.bc = bc_flags & (LBM_WALL_Y | LBM_WALL_Z);
    c->g.layout = inplace ? lbm::kAANatural : lbm::kPull;
    c->inplace = inplace;
    c->sr32 = sr32;
    c->g.plane = px * ny;
    c->g.pop = px * ny * nz;
    for (int b = 0; b < 27; ++b) c->w[b] = (b >= 4 && b < Q) ? float(omega[b]) : 0.0f;
    for (int i = 0; i < 3; ++i) c->F[i] = force ? float(force[i]) : 0.0f;
    c->cur = 0;
    c->device = dev;
    c->graph_steps = kDefaultGraphSteps;
    c->cuda_error = "";
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *c) {
    if (!c) return;
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->red_scratch) cudaFree(c->red_scratch);
    delete c;
}

size_t lbm_state_bytes(const lbm_ctx *c) {
    if (!c) return 0;
    size_t bytes = size_t(c->Q) * size_t(c->g.pop) * elem_bytes(c->storage);
    // BF16: the momentum references of the stored values, a float4 per pair
    // of cells (8 bytes per cell), two arrays for the in-place scheme
    if (c->storage == LBM_STORE_BF16) bytes += (c->inplace ? 2 : 1) * 8 * size_t(c->g.pop);
    return bytes;
}

int lbm_row_pitch(const lbm_ctx *c) { return c ? c->g.px : 0; }

lbm_status lbm_bind(lbm_ctx *c, void *f_a, void *f_b, const float *force_field) {
    if (c && c->inplace) {
        if (!f_a || f_b || (reinterpret_cast<uintptr_t>(f_a) & 255u)) return LBM_EINVAL;
        if (force_field && (reinterpret_cast<uintptr_t>(force_field) & 3u)) return LBM_EINVAL;
        c->buf[0] = f_a;
        c->buf[1] = nullptr;
        c->cur = 0;
        c->g.layout = lbm::kAANatural;
        c->Ffield = force_field;
        c->bound = true;
        c->state_set = false;
        return LBM_OK;
    }
    if (!c || !f_a || !f_b || f_a == f_b) return LBM_EINVAL;
    if ((reinterpret_cast<uintptr_t>(f_a) | reinterpret_cast<uintptr_t>(f_b)) & 255u)
        return LBM_EINVAL;
    const size_t bytes = lbm_state_bytes(c);
    const char *a = static_cast<const char *>(f_a), *b = static_cast<const char *>(f_b);
    if (a < b + bytes && b < a + bytes) return LBM_EINVAL;  // overlap
    if (force_field && (reinterpret_cast<uintptr_t>(force_field) & 3u)) return LBM_EINVAL;
    c->buf[0] = f_a;
    c->buf[1] = f_b;
    c->cur = 0;
    c->Ffield = force_field;
    c->bound = true;
    c->state_set = false;
    return LBM_OK;
}

lbm_status lbm_set_force(lbm_ctx *c, const double *force) {
    if (!c) return LBM_EINVAL;
    if (force)
        for (int i = 0; i < 3; ++i)
            if (!std::isfinite(force[i])) return LBM_EINVAL;
    for (int i = 0; i < 3; ++i) c->F[i] = force ? float(force[i]) : 0.0f;
    return LBM_OK;
}

lbm_status lbm_set_force_field(lbm_ctx *c, const float *force_field) {
    if (!c) return LBM_EINVAL;
    if (force_field && (reinterpret_cast<uintptr_t>(force_field) & 3u)) return LBM_EINVAL;
    c->Ffield = force_field;
    return LBM_OK;
}

lbm_status lbm_set_omega(lbm_ctx *c, const double *omega) {
    if (!c || !valid_rates(c->Q, omega)) return LBM_EINVAL;
    for (int b = 4; b < c->Q; ++b) c->w[b] = float(omega[b]);
    return LBM_OK;
}

lbm_status lbm_init_equilibrium(lbm_ctx *c, const double *rho, const double *u, void *stream) {
    if (!c || !rho || !u) return LBM_EINVAL;
    if (!c->bound) return LBM_ESTATE;
    if (c->inplace) c->g.layout = lbm::kAANatural;
    const lbm::StepArgs a = step_args(c);
    cudaError_t e = dispatch<InitFn>(c, c->buf[c->cur], a, rho, u, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->state_set = true;
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_ctx *c, const double *f, void *stream) {
    if (!c || !f) return LBM_EINVAL;
    if (!c->bound) return LBM_ESTATE;
    if (c->inplace) c->g.layout = lbm::kAANatural;
    cudaError_t e = dispatch<SetFn>(c, c->buf[c->cur], c->g, f, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->state_set = true;
    return LBM_OK;
}

lbm_status lbm_get_state(const lbm_ctx *c, double *f, void *stream) {
    if (!c || !f) return LBM_EINVAL;
    if (!c->bound || !c->state_set) return LBM_ESTATE;
    cudaError_t e = dispatch<GetFn>(c, (const void *)c->buf[c->cur], c->g, f,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return LBM_OK;
}

// Enqueue n step launches on st, advancing the state parity in c.
static cudaError_t enqueue_steps(lbm_ctx *c, int n, cudaStream_t st) {
    for (int s = 0; s < n; ++s) {
        const lbm::StepArgs a = step_args(c);
        cudaError_t e;
        if (c->inplace) {
            const bool even = c->g.layout == lbm::kAANatural;
            e = dispatch<StepAAFn>(c, c->buf[0], a, even, st);
            c->g.layout = even ? lbm::kAASwapped : lbm::kAANatural;
        } else {
            e = dispatch<StepFn>(c, (const void *)c->buf[c->cur], c->buf[1 - c->cur], a, st);
            c->cur = 1 - c->cur;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The graph of c->graph_steps steps from the current arguments and parity,
// captured on first use.  nullptr if capturing failed (the caller then
// launches step by step; the failure leaves no error state behind).
static StepGraph *graph_for(lbm_ctx *c) {
    const GraphKey k = graph_key(c, c->graph_steps);
    StepGraph *slot = &c->graphs[0];
    for (StepGraph &g : c->graphs) {
        if (g.exec && std::memcmp(&g.key, &k, sizeof(k)) == 0) {
            g.used = ++c->graph_clock;
            return &g;
        }
        if (g.used < slot->used) slot = &g;
    }
    if (!c->cap_stream &&
        cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->cap_stream = nullptr;
        return nullptr;
    }
    if (slot->exec) cudaGraphExecDestroy(slot->exec);
    slot->exec = nullptr;
    slot->used = 0;
    // capture with a copy of the parity: the capture launches nothing
    const int cur = c->cur, layout = c->g.layout;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t el = enqueue_steps(c, c->graph_steps, c->cap_stream);
        e = cudaStreamEndCapture(c->cap_stream, &graph);
        if (e == cudaSuccess) e = el;
    }
    c->cur = cur;
    c->g.layout = layout;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    slot->key = k;
    slot->exec = exec;
    slot->used = ++c->graph_clock;
    return slot;
}

lbm_status lbm_step(lbm_ctx *c, int nsteps, void *stream) {
    if (!c || nsteps < 0) return LBM_EINVAL;
    if (!c->bound || !c->state_set) return LBM_ESTATE;
    cudaStream_t st = (cudaStream_t)stream;
    int left = nsteps;
    if (c->graph_steps > 0 && left >= c->graph_steps) {
        // inside a caller's own stream capture, launch step by step
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
            cudaGetLastError();
            cs = cudaStreamCaptureStatusActive;
        }
        while (cs == cudaStreamCaptureStatusNone && left >= c->graph_steps) {
            StepGraph *g = graph_for(c);
            if (!g) break;
            const cudaError_t e = cudaGraphLaunch(g->exec, st);
            if (e != cudaSuccess) return cuda_fail(c, e);
            left -= c->graph_steps;  // an even count: the parity is unchanged
        }
    }
    const cudaError_t e = enqueue_steps(c, left, st);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return LBM_OK;
}

lbm_status lbm_set_graph_steps(lbm_ctx *c, int steps) {
    if (!c || steps < 0 || steps % 2 != 0) return LBM_EINVAL;
    if (steps != c->graph_steps) drop_graphs(c);
    c->graph_steps = steps;
    return LBM_OK;
}

lbm_status lbm_macroscopic(const lbm_ctx *c, float *rho, float *u, void *stream) {
    if (!c) return LBM_EINVAL;
    if (!c->bound || !c->state_set) return LBM_ESTATE;
    if (!rho && !u) return LBM_OK;
    const lbm::StepArgs a = step_args(c);
    cudaError_t e =
        dispatch<MacroFn>(c, (const void *)c->buf[c->cur], a, rho, u, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return LBM_OK;
}

static lbm_status ensure_scratch(lbm_ctx *c, int blocks) {
    if (!c->red_scratch || c->red_blocks < blocks) {
        if (c->red_scratch) cudaFree(c->red_scratch);
        c->red_scratch = nullptr;
        c->red_blocks = 0;
        if (cudaMalloc(&c->red_scratch, sizeof(double) * (4 * size_t(blocks) + 4)) !=
            cudaSuccess) {
            cudaGetLastError();
            return LBM_ENOMEM;
        }
        c->red_blocks = blocks;
    }
    return LBM_OK;
}

lbm_status lbm_conservation(lbm_ctx *c, double out[4], void *stream) {
    if (!c || !out) return LBM_EINVAL;
    if (!c->bound || !c->state_set) return LBM_ESTATE;
    const long long N = (long long)c->g.nx * c->g.ny * c->g.nz;
    const int blocks = lbm::conservation_blocks(c->g);
    const lbm_status ms = ensure_scratch(c, blocks);
    if (ms != LBM_OK) return ms;
    const lbm::StepArgs a = step_args(c);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = dispatch<ConsFn>(c, (const void *)c->buf[c->cur], a, c->red_scratch, blocks, s);
    if (e != cudaSuccess) return cuda_fail(c, e);
    double *tot = c->red_scratch + 4 * size_t(c->red_blocks);
    e = lbm::launch_reduce_final(c->red_scratch, blocks, tot, s);
    if (e != cudaSuccess) return cuda_fail(c, e);
    double h[4];
    e = cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e);
    out[0] = double(N) + h[0];  // the rest state carries mass 1 per cell
    out[1] = h[1];
    out[2] = h[2];
    out[3] = h[3];
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(out[k])) return LBM_ENONFINITE;
    return LBM_OK;
}

size_t lbm_adjoint_bytes(const lbm_ctx *c) {
    if (!c) return 0;
    return size_t(c->Q) * size_t(c->g.pop) * sizeof(float);
}

const void *lbm_current_state(const lbm_ctx *c) {
    if (!c || !c->bound || !c->state_set || c->inplace) return nullptr;
    return c->buf[c->cur];
}

static bool state_buffer_ok(const void *p) {
    return p && (reinterpret_cast<uintptr_t>(p) & 255u) == 0;
}

lbm_status lbm_step_into(lbm_ctx *c, const void *f_in, void *f_out, void *stream) {
    if (!c || !state_buffer_ok(f_in) || !state_buffer_ok(f_out) || f_in == f_out)
        return LBM_EINVAL;
    const size_t bytes = lbm_state_bytes(c);
    const char *a = static_cast<const char *>(f_in), *b = static_cast<const char *>(f_out);
    if (a < b + bytes && b < a + bytes) return LBM_EINVAL;
    if (c->inplace) return LBM_EUNSUPPORTED;
    const lbm::StepArgs args = step_args(c);
    cudaError_t e = dispatch<StepFn>(c, f_in, f_out, args, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return LBM_OK;
}

lbm_status lbm_adjoint_step(lbm_ctx *c, const void *f_t, const float *lam_next, float *lam_out,
                            float *dJdF, void *stream) {
    if (!c || !state_buffer_ok(f_t) || !lam_next || !lam_out || lam_next == lam_out)
        return LBM_EINVAL;
    if ((reinterpret_cast<uintptr_t>(lam_next) | reinterpret_cast<uintptr_t>(lam_out)) & 15u)
        return LBM_EINVAL;
    {
        // the step pulls lam_next from neighbouring cells while writing
        // lam_out: the two fields must not share any byte
        const size_t bytes = lbm_adjoint_bytes(c);
        const char *a = reinterpret_cast<const char *>(lam_next);
        const char *b = reinterpret_cast<const char *>(lam_out);
        if (a < b + bytes && b < a + bytes) return LBM_EINVAL;
    }
    if (dJdF && (reinterpret_cast<uintptr_t>(dJdF) & 3u)) return LBM_EINVAL;
    if (c->inplace) return LBM_EUNSUPPORTED;
    const lbm::StepArgs a = step_args(c);
    cudaError_t e = dispatch<AdjointFn>(c, f_t, lam_next, lam_out, dJdF, a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return LBM_OK;
}

lbm_status lbm_kinetic_energy_seed(lbm_ctx *c, const void *f, float *lam_out, float *dJdF,
                                   void *stream) {
    if (!c || !lam_out) return LBM_EINVAL;
    lbm::StepArgs a = step_args(c);
    if (!f) {
        if (!c->bound || !c->state_set) return LBM_ESTATE;
        f = c->buf[c->cur];
    } else {
        a.g.layout = lbm::kPull;  // a caller's buffer holds a two-buffer state
    }
    if (!state_buffer_ok(f) || (reinterpret_cast<uintptr_t>(lam_out) & 15u)) return LBM_EINVAL;
    if (reinterpret_cast<uintptr_t>(dJdF) & 3u) return LBM_EINVAL;
    cudaError_t e = dispatch<SeedFn>(c, f, lam_out, dJdF, a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return LBM_OK;
}

lbm_status lbm_macroscopic_seed(lbm_ctx *c, const void *f, const float *g_rho, const float *g_u,
                                float *lam_out, float *dJdF, void *stream) {
    if (!c || !lam_out) return LBM_EINVAL;
    lbm::StepArgs a = step_args(c);
    if (!f) {
        if (!c->bound || !c->state_set) return LBM_ESTATE;
        f = c->buf[c->cur];
    } else {
        a.g.layout = lbm::kPull;  // a caller's buffer holds a two-buffer state
    }
    if (!state_buffer_ok(f) || (reinterpret_cast<uintptr_t>(lam_out) & 15u)) return LBM_EINVAL;
    if ((reinterpret_cast<uintptr_t>(g_rho) | reinterpret_cast<uintptr_t>(g_u) |
         reinterpret_cast<uintptr_t>(dJdF)) & 3u)
        return LBM_EINVAL;
    cudaError_t e = dispatch<MacroSeedFn>(c, f, g_rho, g_u, lam_out, dJdF, a,
                                        (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return LBM_OK;
}

lbm_status lbm_kinetic_energy(lbm_ctx *c, const void *f, double *out, void *stream) {
    if (!c || !out) return LBM_EINVAL;
    lbm::StepArgs a = step_args(c);
    if (!f) {
        if (!c->bound || !c->state_set) return LBM_ESTATE;
        f = c->buf[c->cur];
    } else {
        a.g.layout = lbm::kPull;  // a caller's buffer holds a two-buffer state
    }
    if (!state_buffer_ok(f)) return LBM_EINVAL;
    const int blocks = lbm::conservation_blocks(c->g);
    const lbm_status ms = ensure_scratch(c, blocks);
    if (ms != LBM_OK) return ms;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = dispatch<EnergyFn>(c, f, a, c->red_scratch, blocks, s);
    if (e != cudaSuccess) return cuda_fail(c, e);
    double *tot = c->red_scratch + 4 * size_t(c->red_blocks);
    e = lbm::launch_reduce_final(c->red_scratch, blocks, tot, s);
    if (e != cudaSuccess) return cuda_fail(c, e);
    double h[4];
    e = cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e);
    *out = h[0];
    return std::isfinite(h[0]) ? LBM_OK : LBM_ENONFINITE;
}

// ---- conservation sums without any allocation ------------------------------
//
// Some callers cannot let a library call cudaMalloc: codes whose device
// memory is planned once at start-up and handed out from their own pool (an
// allocation by a library would fall outside that plan and can fail once
// the pool holds the device), and loops that cannot afford the device-wide
// synchronisation cudaMalloc and cudaFree may imply.  lbm_conservation
// allocates its reduction scratch on first use; lbm_conservation_noalloc
// keeps the same partial sums in the file-scope array below, which every GPU
// that loads this library holds until the process exits.
//
// The array has room for one partial record (4 doubles) per (y, z) row of
// the grid, for at most kNoAllocMaxRows rows (2 MiB).  Each call launches one
// block per row, each block overwrites its own record, and the final
// reduction reads only the records this call wrote, so no part of the array
// has to start at zero; it keeps the last call's contents.  Calls share the
// array: two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it.
constexpr int kNoAllocMaxRows = 65536;
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) double g_noalloc_part[4 * kNoAllocMaxRows];

namespace {

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kNoAllocMaxDevices];  // device address of the array, per device

// Device address of g_noalloc_part on the current device.  In host code the
// name g_noalloc_part is only a host-side stand-in for the device array, so
// its address is looked up once per device, with that device current.
lbm_status noalloc_scratch(int device, double **out) {
    if (device < 0 || device >= kNoAllocMaxDevices) return LBM_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_part);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return LBM_ECUDA;
        }
        g_noalloc_ptr[device] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[device];
    return LBM_OK;
}
}  // namespace

// Address through which the context's GPU writes the 4 results at `out`:
// device memory of that GPU, managed memory, or page-locked host memory
// mapped into the GPU's address space.  Plain (pageable) host memory and
// another GPU's memory are refused, before anything is launched: a kernel
// writing there would fault.
static lbm_status device_result_ptr(const lbm_ctx *c, double *out, double **dev_out) {
    cudaPointerAttributes at;
    std::memset(&at, 0, sizeof(at));
    if (cudaPointerGetAttributes(&at, out) != cudaSuccess) {
        cudaGetLastError();
        return LBM_EINVAL;
    }
    switch (at.type) {
        case cudaMemoryTypeDevice:
            if (at.device != c->device) return LBM_EINVAL;
            *dev_out = static_cast<double *>(at.devicePointer);
            return *dev_out ? LBM_OK : LBM_EINVAL;
        case cudaMemoryTypeManaged:
            *dev_out = out;
            return LBM_OK;
        case cudaMemoryTypeHost:
            *dev_out = static_cast<double *>(at.devicePointer);  // NULL if not mapped
            return *dev_out ? LBM_OK : LBM_EINVAL;
        default:
            return LBM_EINVAL;
    }
}

lbm_status lbm_conservation_noalloc(lbm_ctx *c, double *out, void *stream) {
    if (!c || !out || (reinterpret_cast<uintptr_t>(out) & 7u)) return LBM_EINVAL;
    if (!c->bound || !c->state_set) return LBM_ESTATE;
    const long long rows = (long long)c->g.ny * c->g.nz;
    if (rows > kNoAllocMaxRows) return LBM_EINVAL;  // grid beyond the array's capacity
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
    if (dev != c->device) return LBM_ESTATE;  // the context's device must be current
    double *dout = nullptr;
    const lbm_status ps = device_result_ptr(c, out, &dout);
    if (ps != LBM_OK) return ps;
    double *part = nullptr;
    const lbm_status st = noalloc_scratch(dev, &part);
    if (st != LBM_OK) return st;
    const lbm::StepArgs a = step_args(c);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = dispatch<ConsFn>(c, (const void *)c->buf[c->cur], a, part, int(rows), s);
    if (e != cudaSuccess) return cuda_fail(c, e);
    e = lbm::launch_reduce_final(part, int(rows), dout, s);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return LBM_OK;
}

const char *lbm_status_string(lbm_status s) {
    switch (s) {
        case LBM_OK: return "LBM_OK";
        case LBM_EINVAL: return "LBM_EINVAL: invalid argument";
        case LBM_ENOMEM: return "LBM_ENOMEM: allocation failed";
        case LBM_ESTATE: return "LBM_ESTATE: call out of order";
        case LBM_ECUDA: return "LBM_ECUDA: CUDA error";
        case LBM_ENONFINITE: return "LBM_ENONFINITE: non-finite conservation sum";
        case LBM_EUNSUPPORTED: return "LBM_EUNSUPPORTED: not provided by this build";
        default: return "unknown lbm_status";
    }
}

const char *lbm_last_cuda_error(const lbm_ctx *c) { return c ? c->cuda_error : ""; }

}  // extern "C"
