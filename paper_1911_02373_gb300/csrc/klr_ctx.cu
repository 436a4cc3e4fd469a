// Context, scratch memory, errors, bases and the configuration set F.
#include <cstdarg>
#include <cstring>
#include <vector>
#include <algorithm>
#include <array>

#include "klr_common.cuh"

namespace klr {

static thread_local char g_error[512] = "no error";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_error, sizeof(g_error), fmt, ap);
    va_end(ap);
}

klr_status ensure_workspace(Context* ctx, size_t bytes, cudaStream_t stream) {
    if (bytes <= ctx->ws_bytes) return KLR_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    KLR_CHECK_CUDA(cudaStreamIsCapturing(stream, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
        set_error("scratch memory of %zu bytes needed during graph capture (have %zu); "
                  "call klr_ctx_reserve first", bytes, ctx->ws_bytes);
        return KLR_ENOMEM;
    }
    KLR_CHECK_CUDA(cudaStreamSynchronize(stream));
    if (ctx->ws) KLR_CHECK_CUDA(cudaFree(ctx->ws));
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    size_t want = std::max(bytes, (size_t)1 << 20);
    if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu bytes of scratch failed", want);
        return KLR_ENOMEM;
    }
    ctx->ws_bytes = want;
    return KLR_OK;
}

uint64_t tune_key(int op, std::initializer_list<int64_t> parts) {
    // FNV-1a over the parts
    uint64_t h = 1469598103934665603ull ^ (uint64_t)op;
    h *= 1099511628211ull;
    for (int64_t p : parts) {
        for (int i = 0; i < 8; ++i) {
            h ^= (uint64_t)((p >> (8 * i)) & 0xff);
            h *= 1099511628211ull;
        }
    }
    return h;
}

int32_t tune_choice(const Context* c, uint64_t key, int32_t dflt) {
    if (c->forced >= 0) return c->forced;
    for (const auto& e : c->tuned)
        if (e.first == key) return e.second;
    return dflt;
}

void tune_store(Context* c, uint64_t key, int32_t choice) {
    for (auto& e : c->tuned)
        if (e.first == key) { e.second = choice; return; }
    c->tuned.emplace_back(key, choice);
}

int log2_bucket(int64_t v) {
    int b = 0;
    while (v > 1) { v >>= 1; ++b; }
    return b;
}

klr_status tune_candidates(Context* c, uint64_t key, cudaStream_t stream, const int32_t* cand,
                           int n_cand, int reps, const std::function<klr_status()>& run,
                           int32_t* choice_out, float* ms_out) {
    KLR_REQUIRE(n_cand > 0 && reps > 0, "autotune: no candidates");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    KLR_CHECK_CUDA(cudaStreamIsCapturing(stream, &cs));
    KLR_REQUIRE(cs == cudaStreamCaptureStatusNone,
                "autotune: the stream is capturing a graph (tune before capturing)");
    cudaEvent_t e0, e1;
    KLR_CHECK_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        set_error("autotune: cudaEventCreate failed");
        return KLR_ECUDA;
    }
    klr_status st = KLR_OK;
    int32_t best = cand[0];
    float best_ms = INFINITY;
    for (int i = 0; i < n_cand && st == KLR_OK; ++i) {
        c->forced = cand[i];
        st = run();                                   // warm-up (and scratch sizing)
        if (st != KLR_OK) break;
        if (cudaEventRecord(e0, stream) != cudaSuccess) {
            set_error("autotune: cudaEventRecord failed");
            st = KLR_ECUDA;
            break;
        }
        for (int r = 0; r < reps && st == KLR_OK; ++r) st = run();
        if (st != KLR_OK) break;
        float ms = 0.f;
        if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            set_error("autotune: timing a candidate failed");
            st = KLR_ECUDA;
            break;
        }
        ms /= (float)reps;
        if (ms < best_ms) { best_ms = ms; best = cand[i]; }
    }
    c->forced = -1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != KLR_OK) return st;
    tune_store(c, key, best);
    if (choice_out) *choice_out = best;
    if (ms_out) *ms_out = best_ms;
    return run();
}

int n_monomials(int n_vars, int degree) {
    // C(n_vars + degree, degree)
    long r = 1;
    for (int i = 1; i <= degree; ++i) r = r * (n_vars + i) / i;
    return (int)r;
}

bool make_basis(int n_vars, int degree, const int32_t* var_degree, Basis* b) {
    const bool box = var_degree && var_degree[0] > 0;
    if (n_vars < 1 || n_vars > kMaxVars) return false;
    if (!box && (degree < 0 || degree > 3)) return false;
    if (box)
        for (int v = 0; v < n_vars; ++v)
            if (var_degree[v] < 0 || var_degree[v] > 3) return false;
    std::memset(b, 0, sizeof(*b));
    b->n_vars = n_vars;
    b->box = box ? 1 : 0;
    // graded: for each total degree, exponent tuples in decreasing lex order
    struct Rec {
        static void go(int pos, int left, std::vector<int>& cur,
                       std::vector<std::vector<int>>& out) {
            int nv = (int)cur.size();
            if (pos == nv - 1) {
                cur[pos] = left;
                out.push_back(cur);
                return;
            }
            for (int v = left; v >= 0; --v) {
                cur[pos] = v;
                go(pos + 1, left - v, cur, out);
            }
        }
    };
    int top = 2 * degree;
    if (box) {
        top = 0;
        for (int v = 0; v < n_vars; ++v) top += 2 * var_degree[v];
    }
    auto within = [&](const std::vector<int>& t, int scale) {
        if (!box) return true;
        for (int v = 0; v < n_vars; ++v)
            if (t[v] > scale * var_degree[v]) return false;
        return true;
    };
    std::vector<std::vector<int>> basis, rest;
    for (int d = 0; d <= top; ++d) {
        std::vector<std::vector<int>> level;
        std::vector<int> cur(n_vars, 0);
        Rec::go(0, d, cur, level);
        for (auto& t : level) {
            const bool in_basis = box ? within(t, 1) : d <= degree;
            if (in_basis) basis.push_back(t);
            else if (within(t, 2)) rest.push_back(t);
        }
    }
    std::vector<std::vector<int>> list = basis;
    for (auto& t : rest) list.push_back(t);
    b->m = (int)basis.size();
    b->degree = degree;
    b->d_n = 0;
    for (auto& t : basis) {
        int s = 0;
        for (int v = 0; v < n_vars; ++v) s += t[v];
        if (box) b->degree = std::max(b->degree, s);
        b->d_n = std::max(b->d_n, t[0]);
    }
    if (box) b->degree = std::min(b->degree, 3);
    b->n_mom = (int)list.size();
    if (b->n_mom > kMaxMoments || b->m > kMaxBasis) return false;
    for (int i = 0; i < b->n_mom; ++i)
        for (int v = 0; v < n_vars; ++v) b->exps[i][v] = (uint8_t)list[i][v];
    for (int i = 0; i < b->m; ++i)
        for (int j = 0; j < b->m; ++j) {
            int found = -1;
            for (int k = 0; k < b->n_mom && found < 0; ++k) {
                bool eq = true;
                for (int v = 0; v < n_vars; ++v)
                    if (list[k][v] != list[i][v] + list[j][v]) eq = false;
                if (eq) found = k;
            }
            b->pair[i][j] = (uint8_t)found;
        }
    return true;
}

}  // namespace klr

using namespace klr;

extern "C" {

const char* klr_last_error(void) { return g_error; }

int klr_version(void) { return KLR_VERSION_MAJOR * 100 + KLR_VERSION_MINOR; }

klr_status klr_ctx_create(klr_ctx** out, int device) {
    KLR_REQUIRE(out != nullptr, "klr_ctx_create: out is NULL");
    int n = 0;
    KLR_CHECK_CUDA(cudaGetDeviceCount(&n));
    KLR_REQUIRE(device >= 0 && device < n, "klr_ctx_create: device %d of %d", device, n);
    KLR_CHECK_CUDA(cudaSetDevice(device));
    Context* c = new Context();
    c->device = device;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) {
        delete c;
        set_error("cudaGetDeviceProperties failed");
        return KLR_ECUDA;
    }
    c->n_sm = p.multiProcessorCount;
    c->smem_optin = p.sharedMemPerBlockOptin;
    *out = reinterpret_cast<klr_ctx*>(c);
    return KLR_OK;
}

klr_status klr_ctx_destroy(klr_ctx* ctx) {
    if (!ctx) return KLR_OK;
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->ws) cudaFree(c->ws);
    delete c;
    return KLR_OK;
}

// Scratch needed by the library for `max_fits` fits and `max_queries` queries.
size_t klr_workspace_bytes(int64_t max_fits, int64_t max_queries);

klr_status klr_tune_export(klr_ctx* ctx, uint64_t* keys, int32_t* choices, int cap, int* n_out) {
    KLR_REQUIRE(ctx != nullptr && n_out != nullptr, "klr_tune_export: NULL argument");
    KLR_REQUIRE(cap >= 0 && (cap == 0 || (keys && choices)), "klr_tune_export: bad buffers");
    const Context* c = reinterpret_cast<const Context*>(ctx);
    const int n = (int)c->tuned.size();
    for (int i = 0; i < n && i < cap; ++i) {
        keys[i] = c->tuned[i].first;
        choices[i] = c->tuned[i].second;
    }
    *n_out = n;
    return KLR_OK;
}

klr_status klr_tune_import(klr_ctx* ctx, const uint64_t* keys, const int32_t* choices, int n) {
    KLR_REQUIRE(ctx != nullptr && n >= 0 && (n == 0 || (keys && choices)),
                "klr_tune_import: bad arguments");
    for (int i = 0; i < n; ++i)
        KLR_REQUIRE(choices[i] >= 0 && choices[i] <= 0xff, "klr_tune_import: choice %d out of range",
                    choices[i]);
    Context* c = reinterpret_cast<Context*>(ctx);
    for (int i = 0; i < n; ++i) tune_store(c, keys[i], choices[i]);
    return KLR_OK;
}

klr_status klr_ctx_reserve(klr_ctx* ctx, int64_t max_fits, int64_t max_queries) {
    KLR_REQUIRE(ctx != nullptr, "klr_ctx_reserve: ctx is NULL");
    KLR_REQUIRE(max_fits >= 0 && max_queries >= 0, "klr_ctx_reserve: negative size");
    Context* c = reinterpret_cast<Context*>(ctx);
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    klr_status st = ensure_workspace(c, klr_workspace_bytes(max_fits, max_queries), 0);
    if (st != KLR_OK) return st;
    KLR_CHECK_CUDA(cudaDeviceSynchronize());
    return KLR_OK;
}

klr_status klr_enumerate_configs(int dims, int min_threads, int max_threads,
                                 int32_t* cfg_out, int capacity, int* count) {
    KLR_REQUIRE(count != nullptr, "klr_enumerate_configs: count is NULL");
    KLR_REQUIRE(dims >= 1 && dims <= 3, "klr_enumerate_configs: dims %d not in 1..3", dims);
    KLR_REQUIRE(min_threads >= 1 && max_threads >= min_threads && max_threads <= (1 << 20),
                "klr_enumerate_configs: bad thread range [%d, %d]", min_threads, max_threads);
    std::vector<std::array<int32_t, 3>> out;
    int max_e = 0;
    while ((1 << (max_e + 1)) <= max_threads) ++max_e;
    for (int i = 0; i <= max_e; ++i)
        for (int j = 0; j <= (dims >= 2 ? max_e : 0); ++j)
            for (int k = 0; k <= (dims >= 3 ? max_e : 0); ++k) {
                long t = (1L << i) * (1L << j) * (1L << k);
                if (t >= min_threads && t <= max_threads && t % 32 == 0)
                    out.push_back({1 << i, 1 << j, 1 << k});
            }
    std::sort(out.begin(), out.end(), [](const std::array<int32_t, 3>& a,
                                         const std::array<int32_t, 3>& b) {
        long ta = (long)a[0] * a[1] * a[2], tb = (long)b[0] * b[1] * b[2];
        if (ta != tb) return ta < tb;
        if (a[0] != b[0]) return a[0] > b[0];
        if (a[1] != b[1]) return a[1] > b[1];
        return a[2] > b[2];
    });
    *count = (int)out.size();
    if (cfg_out) {
        KLR_REQUIRE(capacity >= (int)out.size(),
                    "klr_enumerate_configs: capacity %d < %d", capacity, (int)out.size());
        for (size_t r = 0; r < out.size(); ++r)
            for (int d = 0; d < 3; ++d) cfg_out[3 * r + d] = out[r][d];
    }
    return KLR_OK;
}

}  // extern "C"
