// A group of graph-driven CG solves on one gauge field that share their link
// loads.
//
// Requests of the serving queue that use the same gauge, inner precision and
// inner link format iterate together: each of the four even-odd hops of an
// iteration is one launch of a shared-link kernel over all active members
// (the links of 32 sites staged once in shared memory and applied to every
// member's field, as in the multi right-hand-side kernel), and each BLAS step
// is one launch with a row of blocks per member.  A member keeps its own
// workspace (a GSolve's fields, scalars and reduction scratch); the group only
// holds a device table of the members' pointers and masses.  Per member the
// arithmetic is the same whatever the other members are: its hops read only
// its own fields and the shared links, and its reductions use its own scratch
// with a grid that depends on the lattice only, so a solve gives the same
// bits alone and in any group.
//
// The group's graph is a device-side WHILE loop over iterations, as in
// gsolve.cuh, that stops when any member needs its FP64 reliable update (or
// has converged, broken down or reached maxiter) or after GG_LAUNCH_CAP
// iterations.  The host then takes the members that need an update out of the
// active set (their update runs on their own streams while the others go on)
// and lets members join or rejoin between launches.
#pragma once

#include "dslash_mrhs.cuh"
#include "gsolve.cuh"

namespace wd {

int hop_setup(const wd_gauge *g, int prec, int recon, HopArgs &A);

// Bytes of one half field of precision P (as half_field_bytes).
template <int P> __host__ __device__ constexpr size_t half_bytes_p(int vh) { return Spinor<P>::site_bytes * (size_t)vh; }

constexpr int GG_MAX = 32;          // members of one group at most
constexpr int GG_LAUNCH_CAP = 16;   // iterations at most per group launch

enum { GF_RS = 0, GF_PS = 1, GF_APS = 2, GF_TSO = 3, GF_TSE = 4 };

struct GMember {
    char *f[5];        // rs, ps, aps, tso, tse: inner-precision even/odd half fields
    char *xs;          // FP32 solution increment since the last reliable update
    double *scal;      // the member's CG scalars (see gsolve.cuh)
    RedScratch red;    // its reduction scratch
    double ma, mc;     // m + 4 and -1 / (4 (m + 4)): the Mhat epilogue of its mass
};

struct GTable {
    int n;                 // members in this launch
    int launch_iters;      // iterations run in this launch (reset by the host)
    int idx[GG_MAX];       // their member slots
    GMember m[GG_MAX];     // by slot
};

// ---- shared-link hop over the active members --------------------------------
// Even-odd hop of output parity A.parity0 for every active member: out = f[fo],
// in = f[fi], and with HAS_X the Mhat epilogue out = ma x + mc acc (x = f[fx]);
// without, out = acc.  blockDim = (32, RY): warp y takes members y, y + RY, ...
template <int P, int RECON, bool DAG, bool HAS_X>
__global__ void __launch_bounds__(128, P == PREC_F64 ? 1 : 6)
    hop_group_kernel(const HopArgs A, const GTable *__restrict__ T, const int fi, const int fx, const int fo)
{
    grid_dependency_enter();
    using T_ = typename Prec<P>::real;
    using LT = LinkTile<T_>;
    __shared__ typename LT::V lk[8][LT::NV][32];
    __shared__ int nbs[9][32];
    const int n = T->n;
    if (n == 0) return;
    const int p = A.parity0;
    const int vh = A.vh;
    const int s = threadIdx.x;
    const int i0 = blockIdx.x * 32 + s;
    const bool active = i0 < vh;
    const int i = active ? i0 : -1;
    const char *gf = p ? A.gauge[1] : A.gauge[0];
    const char *gb = p ? A.gauge[0] : A.gauge[1];
    const size_t lb = A.link_blk;
    using LK = Link<link_prec(P), RECON>;
    if (threadIdx.y == 0) {
        nbs[8][s] = i;
        if (active) {
            int nb[8];
            site_neighbours(A, p, i, nb);
#pragma unroll
            for (int d = 0; d < 8; ++d) nbs[d][s] = nb[d];
        }
    }
    __syncthreads();
    const int tid = threadIdx.y * 32 + threadIdx.x, nthr = 32 * blockDim.y;
    for (int pr = tid; pr < 256; pr += nthr) {
        const int d = pr >> 5, ss = pr & 31;
        const int is = nbs[8][ss];
        if (is < 0) continue;
        const int mu = d & 3;
        const char *lblk = d < 4 ? gf + mu * lb : gb + mu * lb;
        const int li = d < 4 ? is : nbs[d][ss];
        cpx<T_> U[3][3];
        LK::template load<true>(lblk, vh, li, U);
        tile_put<T_>(&lk[d][0][ss], U);
    }
    __syncthreads();
    if (!active) return;
    const int *nb = &nbs[0][s];
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    for (int r = threadIdx.y; r < n; r += blockDim.y) {
        const GMember &m = T->m[T->idx[r]];
        const char *in = m.f[fi];
        // 16-bit: the member's hop coefficient weights the terms
        const float wt = Prec<P>::scaled && HAS_X ? (float)m.mc : 1.0f;
        cpx<T_> acc[4][3];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[sp][c] = {T_(0), T_(0)};
        hop_dir_smem<P, 0, SB, false>(in, vh, nb[128], &lk[4][0][s], false, acc, wt);
        hop_dir_smem<P, 1, SB, false>(in, vh, nb[160], &lk[5][0][s], false, acc, wt);
        hop_dir_smem<P, 2, SB, false>(in, vh, nb[192], &lk[6][0][s], false, acc, wt);
        hop_dir_smem<P, 3, SB, false>(in, vh, nb[224], &lk[7][0][s], A.tneg && nb[224] > i, acc, wt);
        hop_dir_smem<P, 0, SF, true>(in, vh, nb[0], &lk[0][0][s], false, acc, wt);
        hop_dir_smem<P, 1, SF, true>(in, vh, nb[32], &lk[1][0][s], false, acc, wt);
        hop_dir_smem<P, 2, SF, true>(in, vh, nb[64], &lk[2][0][s], false, acc, wt);
        hop_dir_smem<P, 3, SF, true>(in, vh, nb[96], &lk[3][0][s], A.tneg && nb[96] < i, acc, wt);
        if constexpr (Prec<P>::scaled) {
            store_weighted<P, HAS_X>(HAS_X ? m.f[fx] : nullptr, m.f[fo], vh, i, (float)m.ma, acc);
            continue;
        }
        T_ o[24];
        if constexpr (HAS_X) {
            const T_ a = (T_)m.ma, b = (T_)m.mc;
            Spinor<P>::load(m.f[fx], vh, i, o);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    o[6 * sp + 2 * c] = a * o[6 * sp + 2 * c] + b * acc[sp][c].re;
                    o[6 * sp + 2 * c + 1] = a * o[6 * sp + 2 * c + 1] + b * acc[sp][c].im;
                }
        } else {
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    o[6 * sp + 2 * c] = acc[sp][c].re;
                    o[6 * sp + 2 * c + 1] = acc[sp][c].im;
                }
        }
        Spinor<P>::store(m.f[fo], vh, i, o);
    }
}

// ---- per-member BLAS steps --------------------------------------------------
// Row y of the grid takes the active members y, y + GG_BLAS_ROWS, ...: a
// member's reduction runs over the gridDim.x blocks of its row whatever the
// group's size, and a small group launches no rows of blocks with nothing to do.
constexpr int GG_BLAS_ROWS = 8;

template <int PS> __global__ void __launch_bounds__(BLAS_THREADS) gg_xpay_kernel(const GTable *__restrict__ T, int vh)
{
    grid_dependency_enter();
    const size_t hs = half_bytes_p<PS>(vh);
    for (int t = blockIdx.y; t < T->n; t += gridDim.y) {
        const GMember &m = T->m[T->idx[t]];
        blas_body(OpXpayDev<PS>{FieldRef<PS>{m.f[GF_RS], hs, vh}, FieldRef<PS>{m.f[GF_PS], hs, vh}, m.scal}, vh, m.red);
        __syncthreads();   // the next member reuses blas_body's shared memory
    }
}

template <int PS> __global__ void __launch_bounds__(BLAS_THREADS) gg_dot_kernel(const GTable *__restrict__ T, int vh)
{
    grid_dependency_enter();
    const size_t hs = half_bytes_p<PS>(vh);
    for (int t = blockIdx.y; t < T->n; t += gridDim.y) {
        const GMember &m = T->m[T->idx[t]];
        blas_body(OpDotAlphaDev<PS>{FieldRef<PS>{m.f[GF_PS], hs, vh}, FieldRef<PS>{m.f[GF_APS], hs, vh}, m.scal}, vh,
                  m.red);
        __syncthreads();   // the next member reuses blas_body's shared memory
    }
}

template <int PS> __global__ void __launch_bounds__(BLAS_THREADS) gg_update_kernel(const GTable *__restrict__ T, int vh)
{
    grid_dependency_enter();
    const size_t hs = half_bytes_p<PS>(vh), h32 = half_bytes_p<PREC_F32>(vh);
    for (int t = blockIdx.y; t < T->n; t += gridDim.y) {
        const GMember &m = T->m[T->idx[t]];
        OpCgUpdateDev<PREC_F32, PS> up{OpCgUpdate<PREC_F32, PS>{FieldRef<PREC_F32>{m.xs, h32, vh},
                                                               FieldRef<PS>{m.f[GF_RS], hs, vh},
                                                               FieldRef<PS>{m.f[GF_PS], hs, vh},
                                                               FieldRef<PS>{m.f[GF_APS], hs, vh}, m.scal + 2, nullptr},
                                       m.scal};
        blas_body(up, vh, m.red);
        __syncthreads();   // the next member reuses blas_body's shared memory
    }
}

// The loop condition: each active member's bookkeeping as in gs_control_kernel
// (without the per-launch count, kept once for the group); the loop stops when
// any member stops or the group has run GG_LAUNCH_CAP iterations.  The
// members' scalars are copied to `hs` (GS_NSCAL per active position) for the
// host to read after the launch.
__global__ void gg_control_kernel(GTable *T, double *hs, cudaGraphConditionalHandle cond)
{
    grid_dependency_enter();
    const int t = threadIdx.x;
    const int n = T->n;
    bool stop = false;
    if (t < n) {
        double *s = T->m[T->idx[t]].scal;
        stop = gs_member_step(s);
        for (int k = 0; k < GS_NSCAL; ++k) hs[t * GS_NSCAL + k] = s[k];
    }
    stop = __syncthreads_or(stop);
    if (t == 0) {
        const int li = T->launch_iters + 1;
        T->launch_iters = li;
        cudaGraphSetConditional(cond, (stop || n == 0 || li >= GG_LAUNCH_CAP) ? 0u : 1u);
    }
}

// Host side of a group: its stream, graph and tables.
struct GGroup {
    const wd_gauge *gauge = nullptr;
    int prec = WD_F32, recon = 18;
    cudaStream_t s = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond = 0;
    GTable *d_table = nullptr, *h_table = nullptr;   // device table, pinned host copy
    double *d_hs = nullptr, *h_hs = nullptr;         // members' scalars after a launch
};

namespace gg_detail {

template <int PS> int build(const wd_ctx *ctx, GGroup &g)
{
    HopArgs A{};
    WD_TRY(hop_setup(g.gauge, PS, g.recon, A));
    A.nparity = 1;
    const int vh = A.vh;
    cudaGraph_t graph;
    WD_CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaError_t ge = cudaGraphConditionalHandleCreate(&g.cond, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = g.cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    if (ge == cudaSuccess) ge = cudaGraphAddNode(&loop, graph, nullptr, nullptr, 0, &cp);
    if (ge != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_error(WD_ECUDA, "creating the group loop failed: %s", cudaGetErrorString(ge));
    }
    GraphSink sink;
    sink.graph = cp.conditional.phGraph_out[0];
    graph_sink() = &sink;
    const dim3 bgrid((unsigned)blas_grid(ctx, vh), (unsigned)GG_BLAS_ROWS), bblk(BLAS_THREADS);
    const dim3 hgrid((unsigned)((vh + 31) / 32)), hblk(32, 4);
    const GTable *T = g.d_table;
    HopArgs Ao = A, Ae = A;
    Ao.parity0 = WD_ODD;
    Ae.parity0 = WD_EVEN;
    wd_launch(gg_xpay_kernel<PS>, bgrid, bblk, 0, g.s, T, vh);
    if (g.recon == 12) {
        wd_launch(hop_group_kernel<PS, 12, false, false>, hgrid, hblk, 0, g.s, Ao, T, (int)GF_PS, 0, (int)GF_TSO);
        wd_launch(hop_group_kernel<PS, 12, false, true>, hgrid, hblk, 0, g.s, Ae, T, (int)GF_TSO, (int)GF_PS, (int)GF_TSE);
        wd_launch(hop_group_kernel<PS, 12, true, false>, hgrid, hblk, 0, g.s, Ao, T, (int)GF_TSE, 0, (int)GF_TSO);
        wd_launch(hop_group_kernel<PS, 12, true, true>, hgrid, hblk, 0, g.s, Ae, T, (int)GF_TSO, (int)GF_TSE, (int)GF_APS);
    } else {
        wd_launch(hop_group_kernel<PS, 18, false, false>, hgrid, hblk, 0, g.s, Ao, T, (int)GF_PS, 0, (int)GF_TSO);
        wd_launch(hop_group_kernel<PS, 18, false, true>, hgrid, hblk, 0, g.s, Ae, T, (int)GF_TSO, (int)GF_PS, (int)GF_TSE);
        wd_launch(hop_group_kernel<PS, 18, true, false>, hgrid, hblk, 0, g.s, Ao, T, (int)GF_TSE, 0, (int)GF_TSO);
        wd_launch(hop_group_kernel<PS, 18, true, true>, hgrid, hblk, 0, g.s, Ae, T, (int)GF_TSO, (int)GF_TSE, (int)GF_APS);
    }
    wd_launch(gg_dot_kernel<PS>, bgrid, bblk, 0, g.s, T, vh);
    wd_launch(gg_update_kernel<PS>, bgrid, bblk, 0, g.s, T, vh);
    wd_launch(gg_control_kernel, dim3(1), dim3(GG_MAX), 0, g.s, g.d_table, g.d_hs, g.cond);
    graph_sink() = nullptr;
    if (sink.err != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_error(WD_ECUDA, "building the group graph failed: %s", cudaGetErrorString(sink.err));
    }
    cudaError_t ce = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return set_error(WD_ECUDA, "group graph instantiation failed: %s", cudaGetErrorString(ce));
    return WD_OK;
}

} // namespace gg_detail

// Allocates a group's stream and tables and builds its graph.
inline int gg_create(const wd_ctx *ctx, GGroup &g)
{
    WD_CUDA_TRY(cudaStreamCreateWithFlags(&g.s, cudaStreamNonBlocking));
    if (cudaMalloc(&g.d_table, sizeof(GTable)) != cudaSuccess ||
        cudaMalloc(&g.d_hs, sizeof(double) * GG_MAX * GS_NSCAL) != cudaSuccess) {
        cudaGetLastError();
        return set_error(WD_ENOMEM, "allocation of a request group's tables failed");
    }
    WD_CUDA_TRY(cudaMallocHost(&g.h_table, sizeof(GTable)));
    WD_CUDA_TRY(cudaMallocHost(&g.h_hs, sizeof(double) * GG_MAX * GS_NSCAL));
    std::memset(g.h_table, 0, sizeof(GTable));
    WD_CUDA_TRY(cudaMemsetAsync(g.d_table, 0, sizeof(GTable), g.s));
    WD_GS_DISPATCH(g.prec, gg_detail::build<PS>(ctx, g));
}

inline void gg_destroy(GGroup &g)
{
    if (g.s) cudaStreamSynchronize(g.s);
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.s) cudaStreamDestroy(g.s);
    cudaFree(g.d_table);
    cudaFree(g.d_hs);
    if (g.h_table) cudaFreeHost(g.h_table);
    if (g.h_hs) cudaFreeHost(g.h_hs);
    g = GGroup{};
}

// The member entry of a bound GSolve.
inline GMember gg_member(const GSolve &q)
{
    GMember m{};
    m.f[GF_RS] = q.rs;
    m.f[GF_PS] = q.ps;
    m.f[GF_APS] = q.aps;
    m.f[GF_TSO] = q.tso;
    m.f[GF_TSE] = q.tse;
    m.xs = q.xs;
    m.scal = q.scal;
    m.red = q.red;
    m.ma = q.mass + 4.0;
    m.mc = -1.0 / (4.0 * (q.mass + 4.0));
    return m;
}

// Enqueues one launch of the group with the members at `slots` (the table
// entries of those slots must be current in h_table), then the copy of their
// scalars to h_hs.
inline int gg_launch(GGroup &g, const int *slots, int n)
{
    g.h_table->n = n;
    g.h_table->launch_iters = 0;
    for (int k = 0; k < n; ++k) g.h_table->idx[k] = slots[k];
    WD_CUDA_TRY(cudaMemcpyAsync(g.d_table, g.h_table, sizeof(GTable), cudaMemcpyHostToDevice, g.s));
    WD_CUDA_TRY(cudaGraphLaunch(g.exec, g.s));
    WD_CUDA_TRY(cudaMemcpyAsync(g.h_hs, g.d_hs, sizeof(double) * GS_NSCAL * n, cudaMemcpyDeviceToHost, g.s));
    return WD_OK;
}

} // namespace wd
