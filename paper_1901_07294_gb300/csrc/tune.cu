// Autotuner for the hop kernel's launch shape and memory schedule.
//
// For one problem (precision, link storage, full or even-odd, with or
// without the axpby term, nrhs, lattice) the tuner times every candidate
// (threads per block x memory-schedule variant) with CUDA events on private
// scratch fields and keeps the fastest in the context.  Later hop launches
// with the same key use it.  With WD_TUNE_CACHE=<file> in the environment the
// results are appended to that file and read back by new contexts.
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <string>

#include "dslash_launch.cuh"
#include "wd_internal.h"

namespace wd {

int hop_setup(const wd_gauge *g, int prec, int recon, HopArgs &A);
std::string hop_key(const wd_ctx *ctx, const HopArgs &A, int prec, int recon, int nrhs);
int hop_launch_cfg(const HopArgs &A, int prec, int recon, int dagger, int nrhs, int threads, int variant,
                   cudaStream_t s);

std::pair<int, int> tuned_config(wd_ctx *ctx, const std::string &key, std::pair<int, int> def)
{
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    auto it = ctx->tuned.find(key);
    return it == ctx->tuned.end() ? def : it->second;
}

// File format: one line per entry, "<threads> <variant> <ms> <key...>".
void load_tune_file(wd_ctx *ctx)
{
    const char *path = std::getenv("WD_TUNE_CACHE");
    if (!path || !*path) return;
    ctx->tune_file = path;
    std::ifstream in(path);
    std::string line;
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    while (std::getline(in, line)) {
        std::istringstream ss(line);
        int threads, variant;
        double ms;
        if (!(ss >> threads >> variant >> ms)) continue;
        std::string key;
        std::getline(ss, key);
        if (!key.empty() && key[0] == ' ') key.erase(0, 1);
        if (threads >= 32 && threads <= 256 && !(threads & 31) && variant >= 0 && variant <= HOP_MAX_VARIANT &&
            variant != HOP_RETIRED_VARIANT)
            ctx->tuned[key] = {threads, variant};
    }
}

} // namespace wd

using namespace wd;

extern "C" {

int wd_tune_dslash(wd_ctx *ctx, const wd_gauge *g, int prec, int recon, int full, int with_x, int nrhs,
                   wd_tune_entry *table, int table_len, int *n_out)
{
    clear_error();
    if (!ctx || !g) return set_error(WD_EINVAL, "NULL argument");
    if (nrhs < 1) return set_error(WD_EINVAL, "nrhs must be >= 1");
    DeviceGuard dg(ctx->device);
    HopArgs A{};
    WD_TRY(hop_setup(g, prec, recon, A));
    const size_t half = half_field_bytes(A.vh, prec);
    const size_t field = (full ? 2 : 1) * half * (size_t)nrhs;
    char *in = nullptr, *out = nullptr, *x = nullptr;
    if (cudaMalloc(&in, field) != cudaSuccess || cudaMalloc(&out, field) != cudaSuccess ||
        (!full && with_x && cudaMalloc(&x, field) != cudaSuccess)) {
        cudaGetLastError();
        cudaFree(in);
        cudaFree(out);
        return set_error(WD_ENOMEM, "cudaMalloc of tuning fields failed");
    }
    cudaStream_t s;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaMemsetAsync(in, 0, field, s);
    if (x) cudaMemsetAsync(x, 0, field, s);
    if (full) {
        for (int p = 0; p < 2; ++p) {
            A.in[p] = in + (size_t)(1 - p) * half;
            A.x[p] = in + (size_t)p * half;
            A.out[p] = out + (size_t)p * half;
        }
        A.rhs_stride = 2 * half;
        A.nparity = 2;
        A.a = 4.1;
        A.b = -0.5;
    } else {
        A.in[0] = A.in[1] = in;
        A.x[0] = A.x[1] = x;
        A.out[0] = A.out[1] = out;
        A.rhs_stride = half;
        A.nparity = 1;
        A.parity0 = 0;
        A.a = 1.0;
        A.b = 1.0;
    }
    const std::string key = hop_key(ctx, A, prec, recon, nrhs);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int cand_threads[] = {64, 128, 192, 256};
    int n = 0, best_t = 256, best_v = 1;
    double best_ms = 1e30;
    int rc = WD_OK;
    for (int ti = 0; ti < 4 && rc == WD_OK; ++ti)
        for (int v = 0; v <= HOP_MAX_VARIANT && rc == WD_OK; ++v) {
            const int th = cand_threads[ti];
            const int zs = hop_mrhs_strip(v);
            if (zs >= 0 && nrhs == 1) continue;
            if (zs > 0 && zs >= A.L[2]) continue;   // same as natural order
            if (v == HOP_RETIRED_VARIANT) continue;
            if ((v == HOP_SP1_VARIANT || v == HOP_SP0_VARIANT) && prec != WD_F16 && prec != WD_BF16) continue;
            if (v == HOP_F64_1B_VARIANT && prec != WD_F64 && prec != WD_DF) continue;
            // double-word FP32: schedules 0 and 1 one block per SM, and the
            // three-threads-per-site kernel (its own block shape: timed once)
            if (prec == WD_DF && v != 0 && v != 1 && v != HOP_F64_1B_VARIANT) continue;
            if (prec == WD_DF && v == HOP_F64_1B_VARIANT && ti > 0) continue;
            for (int w = 0; w < 2 && rc == WD_OK; ++w) rc = hop_launch_cfg(A, prec, recon, 0, nrhs, th, v, s);
            const int reps = 10;
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && rc == WD_OK; ++r) rc = hop_launch_cfg(A, prec, recon, 0, nrhs, th, v, s);
            cudaEventRecord(e1, s);
            cudaError_t ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess && rc == WD_OK) rc = set_error(WD_ECUDA, "tuning run failed: %s", cudaGetErrorString(ce));
            if (rc != WD_OK) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double per = ms / reps;
            if (table && n < table_len) table[n] = wd_tune_entry{th, v, per};
            ++n;
            if (per < best_ms) {
                best_ms = per;
                best_t = th;
                best_v = v;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(in);
    cudaFree(out);
    cudaFree(x);
    if (rc != WD_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        ctx->tuned[key] = {best_t, best_v};
        if (!ctx->tune_file.empty()) {
            FILE *f = std::fopen(ctx->tune_file.c_str(), "a");
            if (f) {
                std::fprintf(f, "%d %d %.6f %s\n", best_t, best_v, best_ms, key.c_str());
                std::fclose(f);
            }
        }
    }
    if (n_out) *n_out = n < table_len ? n : table_len;
    return WD_OK;
}

int wd_tune_set_dslash(wd_ctx *ctx, const wd_gauge *g, int prec, int recon, int full, int with_x, int nrhs,
                       int threads, int variant)
{
    clear_error();
    if (!ctx || !g) return set_error(WD_EINVAL, "NULL argument");
    if (threads < 32 || threads > 256 || (threads & 31) || variant < 0 || variant > HOP_MAX_VARIANT ||
        variant == HOP_RETIRED_VARIANT)
        return set_error(WD_EINVAL, "bad hop launch configuration (%d threads, variant %d)", threads, variant);
    HopArgs A{};
    WD_TRY(hop_setup(g, prec, recon, A));
    A.nparity = full ? 2 : 1;
    static const char dummy = 0;
    A.x[0] = A.x[1] = (full || with_x) ? &dummy : nullptr;
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    ctx->tuned[hop_key(ctx, A, prec, recon, nrhs)] = {threads, variant};
    return WD_OK;
}

int wd_tune_clear(wd_ctx *ctx);

} // extern "C"

namespace wd {

// Tunes one even-odd or full hop shape unless the context already has it.
int hop_ensure_tuned(wd_ctx *ctx, const wd_gauge *g, int prec, int recon, int full, int with_x)
{
    HopArgs A{};
    WD_TRY(hop_setup(g, prec, recon, A));
    A.nparity = full ? 2 : 1;
    static const char dummy = 0;
    A.x[0] = A.x[1] = (full || with_x) ? &dummy : nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        if (ctx->tuned.count(hop_key(ctx, A, prec, recon, 1))) return WD_OK;
    }
    return wd_tune_dslash(ctx, g, prec, recon, full, with_x, 1, nullptr, 0, nullptr);
}

} // namespace wd

extern "C" {

int wd_tune_clear(wd_ctx *ctx)
{
    clear_error();
    if (!ctx) return set_error(WD_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    ctx->tuned.clear();
    return WD_OK;
}

} // extern "C"
