// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "../../include/wdirac.h"

namespace wd {

// Thread-local error message behind wd_last_error().
int set_error(int status, const char *fmt, ...);
void clear_error();

#define WD_CUDA_TRY(expr)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return ::wd::set_error(WD_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                                   __FILE__, __LINE__);                                        \
    } while (0)

#define WD_TRY(expr)                \
    do {                            \
        int s_ = (expr);            \
        if (s_ != WD_OK) return s_; \
    } while (0)

// The solvers stop when their own FP64 true residual |b - A x| / |b| is at most
// SOLVE_TARGET * tol.  Another FP64 evaluation of the same residual (other
// summation order, no FMA) differs from the solver's by the rounding of the
// products in A x, of order u |A| |x| (u = 2^-53, |A| <= 25 for these
// operators).  The 10 % margin covers that whenever u |A| |x| / |b| is well
// below 0.1 tol, so a solve reported converged also meets tol under such a
// re-evaluation.
constexpr double SOLVE_TARGET = 0.9;

struct Geometry {
    int L[4];
    int64_t V;
    int Vh;
};

// Validates dims (all even, >= 2, Vh < 2^31) and fills g.
int make_geometry(const int dims[4], Geometry &g);
bool valid_prec(int prec);         // WD_F64 .. WD_BF16 (solver inner precisions, halos)
bool valid_field_prec(int prec);   // valid_prec or WD_DF (fields, operators, BLAS)
bool valid_recon(int recon);

// Bytes of one half field (one parity) in a storage precision.
size_t half_field_bytes(int vh, int prec);
// Bytes of the links of one (parity, mu) block.
size_t link_block_bytes(int vh, int prec, int recon);

// Restores the calling thread's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

} // namespace wd

struct wd_ctx {
    int device = 0;
    int num_sms = 0;
    int cc_major = 0, cc_minor = 0;
    std::mutex mu;
    // reduction scratch (device): partial sums, a ticket counter and result slots
    double *d_partials = nullptr;
    unsigned *d_ticket = nullptr;
    double *d_scal = nullptr;      // wd::NSCAL result slots
    double *h_scal = nullptr;      // pinned host mirror of d_scal
    // solver workspace (device), grown on demand
    char *d_work = nullptr;
    size_t work_bytes = 0;
    char *d_aux = nullptr;         // second workspace (ctx_aux_workspace)
    size_t aux_bytes = 0;
    // launch-shape cache filled by the autotuner: problem key -> (threads, variant)
    std::mutex tune_mu;
    std::map<std::string, std::pair<int, int>> tuned;
    std::string tune_file;   // on-disk cache (WD_TUNE_CACHE), empty if none
};

struct wd_gauge {
    wd_ctx *ctx = nullptr;         // for tuning lookups; must outlive the gauge's use
    int device = 0;                // kept here so destruction does not need ctx
    wd::Geometry geo{};
    double *canonical = nullptr;   // device, FP64 canonical links (V*4*18 doubles)
    int t_sign = 1;                // +1 periodic in t, -1 antiperiodic
    std::mutex mu;
    std::map<std::pair<int, int>, char *> layouts;  // (prec, recon) -> device buffer
};

namespace wd {
constexpr int NSCAL = 64;
// Device status word of a context: word 32 of the 64-word ticket buffer (word
// 0 is the reduction ticket).  Kernels with bounded waits write their error
// code here; wd_device_status reads and clears it.
inline int *ctx_status_word(const wd_ctx *c) { return c ? reinterpret_cast<int *>(c->d_ticket + 32) : nullptr; }
// Even-odd hop on half fields: out_p = a x_p + b H^(d)_{p,1-p} in (see dslash_eo_apply).
int eo_hop(const wd_gauge *g, int prec, int recon, void *out, const void *in, const void *x, int p, double a,
           double b, int dagger, cudaStream_t s);
// Full-lattice hop on a full field: out = a in + b H in (both parities).
int full_hop(const wd_gauge *g, int prec, int recon, void *out, const void *in, double a, double b, cudaStream_t s);
// Launch configuration of a tunable kernel: the tuned one if the context has
// it, else `def`.
std::pair<int, int> tuned_config(wd_ctx *ctx, const std::string &key, std::pair<int, int> def);
void load_tune_file(wd_ctx *ctx);
// Runs the autotuner for one hop shape unless the context already has it.
int hop_ensure_tuned(wd_ctx *ctx, const wd_gauge *g, int prec, int recon, int full, int with_x);
// Solver workspace of at least `bytes` bytes (device), owned by the context.
int ctx_workspace(wd_ctx *ctx, size_t bytes, char **out);
// A second context-owned device buffer for drivers that call a solver (which
// takes ctx_workspace) and need vectors of their own meanwhile.
int ctx_aux_workspace(wd_ctx *ctx, size_t bytes, char **out);
// The CG solve of cg_solve without its argument checks, locking and timing
// (x, b: FP64 even half fields; the gauge layouts must be prepared).
int cg_dispatch(wd_ctx *ctx, const wd_gauge *g, double mass, char *x, const char *b, double tol,
                const wd_cg_opts &o, wd_cg_stats &st, cudaStream_t s);
// Device pointer of the (prec, recon) layout, built on first use.
int gauge_layout(const wd_gauge *g, int prec, int recon, const char **out);
// Per-(parity, mu) block pointer inside a layout buffer.
inline const char *link_block(const char *base, int vh, int prec, int recon, int parity, int mu)
{
    return base + (size_t)(parity * 4 + mu) * link_block_bytes(vh, prec, recon);
}
} // namespace wd
