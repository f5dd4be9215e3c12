/*
 * wdirac -- Wilson-Dirac operator and solvers on one NVIDIA GB300 (sm_103a).
 *
 * C ABI.  Every function returns a wd_status (0 = success, negative = error)
 * unless stated otherwise; no C++ exception crosses this boundary.  After an
 * error, wd_last_error() returns a message for the calling thread.
 *
 * The operator (arXiv:1901.07294, Sec. II-A, Eq. (1)).  A quark field psi has
 * 4 spin x 3 colour complex components per lattice site; the SU(3) gauge link
 * U_mu(x) sits on the link from x to x+mu.  This library implements the
 * hopping sum
 *     H psi(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                       + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu) ]
 * and the Wilson operator D = (m+4) - H/2, on a periodic 4D lattice, with the
 * Hermitian chiral gamma basis (gamma5 = diag(1,1,-1,-1)).  Eq. (1) as
 * printed (projectors swapped) equals gamma5 H gamma5.
 *
 * Lattice.  dims = {Lx, Ly, Lz, Lt}, every extent even and >= 2; mu = 0..3 =
 * x,y,z,t; lexicographic site = x + Lx*(y + Ly*(z + Lz*t)); parity of a site
 * = (x+y+z+t) mod 2, even = 0.  V = Lx*Ly*Lz*Lt, Vh = V/2 (< 2^31).
 *
 * Canonical (user) layout, FP64, interleaved re/im, lexicographic order:
 *     spinor double[V][4 spin][3 colour][2]
 *     links  double[V][4 mu][3 row][3 col][2]
 *
 * Device field layout (opaque to callers; size from wd_field_bytes()).  A
 * "half field" holds the Vh sites of one parity in checkerboard order
 * cb = site >> 1.  Its 24 reals per site are split into planes of 16-byte
 * vectors (plane-major, site-minor) so that consecutive threads read
 * consecutive 16-byte words:
 *     WD_F64 : 12 planes of double2
 *     WD_F32 :  6 planes of float4
 *     WD_F16, WD_BF16 : 3 planes of 8 halves, then one plane of FP32
 *               per-site scales (stored value = real / scale, scale =
 *               max |real| over the site's 24 reals).
 *     WD_DF  : 12 planes of float4 (hi0, lo0, hi1, lo1): each real is the
 *               unevaluated sum hi + lo of two FP32 numbers with
 *               hi = RN(hi + lo), 48 significand bits.
 * A full field is the even half followed by the odd half.  nrhs > 1 means
 * nrhs fields stored one after another.
 *
 * Memory ownership.  Field pointers are device memory owned by the caller
 * (for example torch tensors); the library never frees them.  Context and
 * gauge objects are owned by the library and released by their destroy call.
 * Pointers passed as fields must be 16-byte aligned.
 *
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).
 * Operator calls are asynchronous on that stream; launch errors are reported
 * at once, asynchronous faults at the next synchronising call.  Kernels are
 * launched with programmatic dependent launch: one may be dispatched while
 * the kernel before it on the stream is finishing, and it waits for that
 * kernel's completion before it reads or writes memory, so stream order holds
 * as for plain launches.  WD_PDL=0 in the environment (read once per process)
 * launches them serialised instead.
 */
#ifndef WDIRAC_H
#define WDIRAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WD_OK = 0,
    WD_EINVAL = -1,      /* bad argument (dims, precision, pointer, alignment) */
    WD_ENOMEM = -2,      /* device or host allocation failed */
    WD_ECUDA = -3,       /* CUDA runtime error */
    WD_ENOCONV = -4,     /* solver reached maxiter without converging */
    WD_ETIMEOUT = -5,    /* a bounded device-side wait gave up */
    WD_ECANCELLED = -6,  /* request cancelled */
    WD_EBUSY = -7        /* result not ready yet */
} wd_status;

/* storage precision; WD_DF (double-word FP32) is a field and operator
 * format, not a solver inner precision or a halo format */
typedef enum { WD_F64 = 0, WD_F32 = 1, WD_F16 = 2, WD_BF16 = 3, WD_DF = 4 } wd_prec;
typedef enum { WD_RECON_18 = 18, WD_RECON_12 = 12 } wd_recon;               /* reals stored per link */
typedef enum { WD_EVEN = 0, WD_ODD = 1 } wd_parity;
typedef enum { WD_SITES_FULL = 0, WD_SITES_EVEN = 1, WD_SITES_ODD = 2 } wd_sites;

typedef struct wd_ctx wd_ctx;
typedef struct wd_gauge wd_gauge;

/* Library version (major*10000 + minor*100 + patch). */
int wd_version(void);

/* Message of the last error on the calling thread ("" if none).  The pointer
 * stays valid until the next wdirac call on this thread. */
const char *wd_last_error(void);

/* Context: binds a CUDA device and holds per-device scratch (reduction
 * partial sums, launch-shape cache).  One context may be shared by threads
 * whose calls do not overlap; give overlapping callers one context each. */
int wd_ctx_create(int device, wd_ctx **out);
int wd_ctx_destroy(wd_ctx *ctx);

/* Bytes of one device field of `sites` (wd_sites) in precision `prec`,
 * times nrhs.  Errors: WD_EINVAL for bad dims, prec or nrhs < 1. */
int wd_field_bytes(const int dims[4], int sites, int prec, int nrhs, size_t *out);

/* Layout conversion (Sec. II-C lists precision conversion among the
 * machine-specific primitives).  wd_pack reads a canonical FP64 spinor of the
 * FULL lattice (V sites) and writes the device field holding `sites` (full,
 * even or odd half) in precision `prec`.  wd_unpack writes the sites held by
 * the field back into a canonical full-lattice array; sites of the other
 * parity are left untouched.  Asynchronous on `stream`.
 * The canonical array may be device memory of the context's GPU, managed
 * memory, page-locked host memory (the kernel then reads or writes it
 * directly over the host link, with no staging copy) or, where the device
 * can access pageable memory (Grace systems), ordinary host memory; anything
 * else gives WD_EINVAL.  The field must be device memory. */
int wd_pack(wd_ctx *ctx, const int dims[4], int sites, int prec, const double *aos,
            void *field, void *stream);
int wd_unpack(wd_ctx *ctx, const int dims[4], int sites, int prec, const void *field,
              double *aos, void *stream);
/* The same with a canonical array of FP32 reals (24 per site, same order): for
 * callers whose host fields are single precision, which halves the bytes that
 * cross the host link for an FP32 or 16-bit workload.  wd_unpack_f32 rounds
 * FP64 fields to FP32. */
int wd_pack_f32(wd_ctx *ctx, const int dims[4], int sites, int prec, const float *aos,
                void *field, void *stream);
int wd_unpack_f32(wd_ctx *ctx, const int dims[4], int sites, int prec, const void *field,
                  float *aos, void *stream);

/* Gauge field (Sec. II-A: one SU(3) matrix per link).  `links` is canonical
 * FP64 (device memory, or host memory if links_on_host != 0); the library
 * keeps its own FP64 copy and builds device layouts on demand: per parity,
 * per mu, planes of 16-byte vectors holding the first `recon` reals of the
 * row-major matrix (12 = rows 0 and 1 only; row 2 is rebuilt in the kernel as
 * conj(row0 x row1), valid for SU(3)).  Synchronous.  Operator calls with a
 * gauge use its context's tuning cache, so the context must outlive those
 * calls; destroying a gauge after its context is allowed. */
int wd_gauge_create(wd_ctx *ctx, const int dims[4], const double *links, int links_on_host,
                    wd_gauge **out);
/* Builds (if not built yet) the (prec, recon) layout.  Operator calls build
 * missing layouts themselves; call this first when the operator call must not
 * allocate (for example before capturing a CUDA graph).  Synchronous. */
int wd_gauge_prepare(wd_gauge *g, int prec, int recon);
/* Boundary condition in t for every operator call with this gauge (and every
 * solve): t_sign = +1 periodic (the default), -1 antiperiodic, i.e. a hop
 * across the t boundary (forward from t = Lt-1, backward from t = 0) changes
 * sign; the same as negating the links U_t on the slice t = Lt-1.  The paper
 * does not fix the boundary conditions; this is the usual fermion choice in
 * time.  Applied in the kernels (the stored links are unchanged).  Must not be
 * called while operator calls or solves with this gauge are in flight.
 * WD_EINVAL unless t_sign is +1 or -1. */
int wd_gauge_set_boundary(wd_gauge *g, int t_sign);
int wd_gauge_bytes(const wd_gauge *g, int prec, int recon, size_t *out);
int wd_gauge_destroy(wd_gauge *g);

/*
 * Full-lattice Wilson-Dirac operator:  out = D in = (m+4) in - H in / 2.
 * `in` and `out` are full fields of precision `prec` (nrhs consecutive
 * fields).  WD_F64 computes in FP64 on FP64 links; WD_F32, WD_F16 and
 * WD_BF16 compute in FP32 on links stored in the field's precision, except
 * that WD_BF16 fields use FP16 links (link entries are bounded by 1, so FP16's
 * 3 extra mantissa bits cost no range).  WD_DF computes in double-word FP32
 * on double-word links (errors of order 2^-48 times the magnitudes of the
 * terms, FP32 instructions only: on a part whose FP64 rate is 1/64 of its
 * FP32 rate it replaces FP64 where 48 bits suffice).  out must not alias in.
 * Flop count: 1320 per site for H (Eq. (1): 8 directions of spin projection,
 * SU(3) x half-spinor and reconstruction).
 */
int dslash_apply(wd_ctx *ctx, const wd_gauge *g, void *out, const void *in, double mass,
                 int nrhs, int prec, int recon, void *stream);

/*
 * out = D^dagger in = gamma5 D gamma5 in = (m+4) in - (gamma5 H gamma5) in / 2.
 * gamma5 H gamma5 is the hopping term of Sec. II-A, Eq. (1) exactly as printed
 * (projector 1 + gamma forward, 1 - gamma backward), so this is also the
 * operator in the paper's sign convention.  Arguments as for dslash_apply.
 */
int dslash_apply_dagger(wd_ctx *ctx, const wd_gauge *g, void *out, const void *in, double mass,
                        int nrhs, int prec, int recon, void *stream);

/*
 * Even-odd hopping block with fused axpby:
 *     out_p = a * x_p + b * H^(d)_{p,1-p} in_{1-p},   p = out_parity,
 * where H_{p,1-p} is H restricted to output sites of parity p (its inputs
 * are the sites of parity 1-p), and H^(d) = H (dagger = 0) or
 * gamma5 H gamma5 (dagger = 1; the projectors 1 -+ gamma swap).  `in`, `x`
 * and `out` are half fields; x may be NULL (then a is ignored).  out must not
 * alias in; it may alias x.  With dagger = 1 the block is the adjoint of the
 * opposite block: (H_{p,1-p})^dagger = gamma5 H_{1-p,p} gamma5.
 */
int dslash_eo_apply(wd_ctx *ctx, const wd_gauge *g, void *out, const void *in, const void *x,
                    int out_parity, double a, double b, int dagger, int nrhs, int prec, int recon,
                    void *stream);

/* Measured FMA throughput of the device (TFLOP/s, one FMA = 2 flops) for
 * prec WD_F64 or WD_F32: the ALU roofline of the FP64 operator, which is
 * bounded by the FP64 units rather than by HBM.  The paper has no
 * counterpart; this is measurement support.  Synchronous, about 0.1 s. */
int wd_probe_fma(wd_ctx *ctx, int prec, double *tflops);

/* Device attributes of the context's GPU, for rooflines: SM count, memory
 * clock (kHz), memory bus width (bits), L2 size (bytes), compute capability,
 * the nominal HBM bandwidth 2 x clock x width / 8 (GB/s; two transfers per
 * clock), and whether kernels can access pageable host memory.  Measurement support; the paper has no counterpart. */
typedef struct {
    int sm_count;
    int mem_clock_khz;
    int mem_bus_bits;
    int l2_bytes;
    int cc_major, cc_minor;
    double nominal_hbm_gbs;
    int pageable_memory_access;   /* 1: kernels may dereference ordinary host memory */
} wd_device_props;

int wd_device_info(const wd_ctx *ctx, wd_device_props *out);

/* Asynchronous device-side status of the context: a kernel whose bounded wait
 * gave up records WD_ETIMEOUT in a context-owned word and skips its output.  wd_device_status waits for all work on the context's device,
 * stores that word (WD_OK if nothing was recorded) in *code and clears it.
 * Returns WD_OK, or WD_ECUDA if the device could not be synchronised. */
int wd_device_status(wd_ctx *ctx, int *code);

/* ---- Autotuning of the operator launches ------------------------------------
 * The hop kernel has tunable launch parameters: threads per block (32..256,
 * multiple of 32) and a memory-schedule variant (0: directions x+,x-,..,t-
 * with no prefetch; 1: backward directions first with the forward links and
 * t-forward neighbour prefetched into L2; 2: as 1 plus the backward links;
 * 4: as 1 compiled for 3 resident blocks of 256 threads per SM; for nrhs > 1
 * also 3: links of 32 sites staged once in shared memory for all nrhs fields,
 * and 5, 6, 7: as 3 with the (z, t) slices visited in z-strips of width 16,
 * 8, 4, which shortens the reuse distance of t-neighbours in L2); and the
 * search's other two dimensions: 8: as 1 with each block's window of nearby
 * neighbour spinors staged in shared memory (tiling on), 9: as 1 with two
 * sites per thread; 11, 12: schedules 0 and 1 with the links loaded
 * without L1 allocation, which suits even-odd hops, where each link is read
 * once per call; 13, 14 (FP16 and BF16 fields only): schedules 1 and 0 (the
 * latter with links loaded without L1 allocation) with the two spin
 * components of each projected half spinor carried as a pair through
 * Blackwell's paired FP32 instructions; variant 10 is retired and refused).
 * wd_tune_dslash times every candidate for one problem shape (full = 1: the
 * dslash_apply shape; full = 0: dslash_eo_apply with (with_x = 1) or without
 * the x term) on private scratch fields (allocated and freed by the call),
 * stores the fastest in the context and, if WD_TUNE_CACHE names a file,
 * appends it there (new contexts read that file).  Up to table_len timings
 * are written to `table`.  Synchronous.  Results of tuned and untuned
 * launches can differ in the last bits (the summation order of the eight
 * directions depends on the variant).  wd_tune_set_dslash pins a
 * configuration; wd_tune_clear forgets all of them. */
typedef struct {
    int threads;
    int variant;
    double ms;   /* mean time per launch */
} wd_tune_entry;

int wd_tune_dslash(wd_ctx *ctx, const wd_gauge *g, int prec, int recon, int full, int with_x, int nrhs,
                   wd_tune_entry *table, int table_len, int *n_out);
int wd_tune_set_dslash(wd_ctx *ctx, const wd_gauge *g, int prec, int recon, int full, int with_x, int nrhs,
                       int threads, int variant);
int wd_tune_clear(wd_ctx *ctx);

/* ---- BLAS-1 on device fields (sites = wd_sites of the field) ----------------
 * Reductions accumulate each site's 24 reals in the field's compute type,
 * then sum sites in FP64 (warp shuffles, per-block partials in the context's
 * scratch, fixed-order final sum), so repeated calls are bitwise identical.
 * `result` is device memory.  Calls on one context must not overlap on the
 * GPU (they share the context's scratch). */
int wd_norm2(wd_ctx *ctx, const int dims[4], int sites, int prec, const void *x, double *result,
             void *stream);                                    /* result[0] = |x|^2 */
int wd_dot(wd_ctx *ctx, const int dims[4], int sites, int prec, const void *a, const void *b,
           double *result, void *stream);                      /* result = <a,b> = sum conj(a) b (re, im) */
int wd_axpby(wd_ctx *ctx, const int dims[4], int sites, int prec, double a, const void *x, double b,
             void *y, void *stream);                           /* y = a x + b y */
int wd_convert(wd_ctx *ctx, const int dims[4], int sites, int prec_out, void *out, int prec_in,
               const void *in, void *stream);                  /* out = in, new storage precision */

/* |x|^2 like wd_norm2, for callers that cannot allocate device memory and so
 * cannot create a wd_ctx: plug-ins whose host framework owns all device
 * memory through a pooling allocator and forbids raw cudaMalloc, and
 * latency-critical loops that cannot afford cudaMalloc's implicit device
 * synchronisation.  The paper has no counterpart; this is an interface
 * convenience.
 * The reduction scratch is a fixed 64 KB array in the library's device code
 * (held by every GPU that loads the library until the process exits); fields
 * of more than 2,097,152 sites (e.g. a full 32^3 x 64 field is the largest
 * such lattice) are rejected with WD_EINVAL.  No cudaMalloc/cudaFree or other
 * allocating call is made.  The first call on a device (and the first after
 * its context was reset) looks up the array's device address with that
 * device current (a host-side lookup, made once per device).  All calls
 * share the one array: calls that overlap on the GPU (other streams, other
 * threads) race and give wrong results.  Results equal wd_norm2's up to FP64
 * summation order.  `result` is device memory. */
int wd_norm2_noalloc(const int dims[4], int sites, int prec, const void *x, double *result,
                     void *stream);

/* ---- Domain decomposition with a halo exchange (Sec. II-A) ----------------
 * Sec. II-A parallelises the hopping term by decomposing the lattice into
 * sub-lattices, one per process; Sec. V uses 16-bit floats only to compress
 * the data exchanged between them.  A wd_dd splits the lattice `dims` along t
 * into nsub slabs of L_t/nsub slices (nsub must divide L_t; the slab extent
 * must be even and >= 2).  Slab k holds its own gauge (the k-th contiguous
 * slice of the canonical links, whose site order has t slowest) and works on
 * its own full fields of the local dimensions (wd_dd_local_dims); pack slab
 * k's field with wd_pack from the k-th slice of a canonical global array.
 * All slabs live on this GPU; the exchange is a device copy into each
 * receiver's own halo buffer, the step that a multi-GPU build replaces by
 * NCCL send/recv.
 *
 * wd_dd_dslash: out[k] = D in[k] for every slab k (D = (m+4) - H/2 of the
 * global lattice): the faces (12-real spin-projected half spinors; backward
 * faces already multiplied by the sender's link) are gathered and exchanged
 * on an internal stream while the interior pass (hops that stay inside a
 * slab) runs on `stream`; the boundary sites then add the halo terms.
 * halo_prec: WD_F64, WD_F32 or WD_F16 (with a per-site FP32 scale) for the
 * exchanged faces, independent of the field precision `prec`.  Asynchronous
 * on `stream`.  out[k] must not alias in[k].  wd_dd_set_boundary: +1
 * periodic, -1 antiperiodic in t (the sign goes on the faces that cross the
 * global boundary).  wd_dd_halo_bytes: bytes of faces exchanged per
 * application (all slabs, both directions and parities). */
typedef struct wd_dd wd_dd;

int wd_dd_create(wd_ctx *ctx, const int dims[4], int nsub, const double *links, int links_on_host, wd_dd **out);
int wd_dd_local_dims(const wd_dd *dd, int dims_out[4]);
int wd_dd_set_boundary(wd_dd *dd, int t_sign);
int wd_dd_halo_bytes(const wd_dd *dd, int halo_prec, size_t *out);
int wd_dd_dslash(wd_dd *dd, void *const *out, const void *const *in, double mass, int prec, int recon,
                 int halo_prec, void *stream);
int wd_dd_destroy(wd_dd *dd);

/* ---- One slab per process (Sec. II-A: one sub-lattice per process) ---------
 * The decomposition of wd_dd with each slab in its own process (on its own
 * GPU): the process creates the wd_slab for its slab index k of nsub, from
 * its own slice of the canonical links (local dims = global dims with
 * L_t / nsub, the k-th contiguous slice of the global array; host or device
 * memory as links_on_host says; the slab keeps its own copy).  One
 * application of D to the global lattice is then, in every process:
 *   wd_slab_gather(in -> send_fwd, send_bwd)   faces into caller-owned device
 *       buffers of wd_slab_face_bytes bytes each: send_fwd (the sites at local
 *       t = 0, (1 - gamma_t) projected) goes to slab k-1, send_bwd (the sites
 *       at local t = T-1, U_t^dagger (1 + gamma_t) projected, times this
 *       slab's own link) goes to slab k+1 (indices mod nsub);
 *   the transport (e.g. NCCL send/recv) delivers them into the neighbours'
 *       own buffers: recv_fwd from slab k+1, recv_bwd from slab k-1;
 *   wd_slab_interior(out = D_local in with the t boundary open), which may
 *       run while the faces are in flight;
 *   wd_slab_boundary(out += the halo terms from recv_fwd, recv_bwd), after
 *       both.
 * Halos as for wd_dd_dslash (WD_F64, WD_F32, WD_F16 with a per-site scale);
 * the face format is private to the library, so both ends must use the same
 * halo_prec.  Antiperiodic t (wd_slab_set_boundary(-1)): the faces that cross
 * the global boundary change sign (slab 0's forward face, slab nsub-1's
 * backward face).  Fields are local full fields (wd_pack with the local
 * dims); every pointer 16-byte aligned; asynchronous on `stream`. */
typedef struct wd_slab wd_slab;

int wd_slab_create(wd_ctx *ctx, const int dims[4], int nsub, int k, const double *links, int links_on_host,
                   wd_slab **out);
int wd_slab_local_dims(const wd_slab *sl, int dims_out[4]);
int wd_slab_set_boundary(wd_slab *sl, int t_sign);
int wd_slab_face_bytes(const wd_slab *sl, int halo_prec, size_t *out);
int wd_slab_gather(wd_slab *sl, const void *in, int prec, int recon, int halo_prec, void *send_fwd, void *send_bwd,
                   void *stream);
int wd_slab_interior(wd_slab *sl, void *out, const void *in, double mass, int prec, int recon, void *stream);
int wd_slab_boundary(wd_slab *sl, void *out, const void *recv_fwd, const void *recv_bwd, int prec, int recon,
                     int halo_prec, void *stream);
int wd_slab_destroy(wd_slab *sl);

/* ---- Element-wise products (Sec. IV examples; Sec. III-D complex forms) ----
 * z_i = f(x_i, y_i[, z_i]) for i < n on device arrays of FP64:
 *   WD_STREAM_REAL_MUL        z = x y        n reals (Sec. IV, real arithmetic)
 *   WD_STREAM_CPLX_MUL        z = x y        n complex numbers stored as
 *   WD_STREAM_CPLX_CONJ_MUL   z = conj(x) y  interleaved (re, im) pairs
 *   WD_STREAM_CPLX_MADD       z = z + x y    (Sec. IV, complex arithmetic; the
 *   WD_STREAM_CPLX_CONJ_MADD  z = z + conj(x) y  FCMLA rotation pairs of III-D)
 * Complex products use FMA: re = fma(xr, yr, -(xi yi)), im = fma(xr, yi, xi yr)
 * (the conjugate forms with -xi), so results can differ from a plain
 * multiply-then-add in the last bit.  Arrays must be 16-byte aligned; z may
 * equal x or y (element-wise in place).  Asynchronous on `stream`; n = 0 is a
 * no-op.  HBM stream kernels: also the calibration of the memory roofline. */
typedef enum {
    WD_STREAM_REAL_MUL = 0,
    WD_STREAM_CPLX_MUL = 1,
    WD_STREAM_CPLX_CONJ_MUL = 2,
    WD_STREAM_CPLX_MADD = 3,
    WD_STREAM_CPLX_CONJ_MADD = 4
} wd_stream_kind;

int wd_stream_mul(wd_ctx *ctx, int kind, size_t n, const double *x, const double *y, double *z, void *stream);

/* ---- Conjugate gradient (Sec. II-A: CG solves the Dirac system) ------------
 * Solves  Mhat^dagger Mhat x = b  on the even sites, where
 *     Mhat = (m+4) - H_eo H_oe / (4(m+4))
 * is the Schur complement of D = (m+4) - H/2 and Mhat^dagger = gamma5 Mhat
 * gamma5.  x_e and b_e are even half fields in WD_F64 (device).  x_0 = 0.
 * Converged when the true residual |b - A x| / |b| <= tol, computed in FP64.
 * inner_prec = WD_F64: plain FP64 CG.  Otherwise mixed precision: the
 * iterated residual, search direction and operator use inner_prec storage
 * (FP32 arithmetic), while the solution, true residual and all inner products
 * are FP64.  reliable = 1: reliable updates (Sleijpen-van der Vorst) when the
 * iterated residual has dropped by `delta` since the last update;
 * reliable = 0: iterative refinement with restarted inner solves to relative
 * residual `delta`.  Synchronous; uses a workspace owned by the context
 * (allocated on first use, grown when a larger lattice needs more).
 * Returns WD_ENOCONV (stats still filled) if maxiter inner iterations pass
 * without convergence or the iteration breaks down. */
typedef struct {
    int inner_prec;    /* wd_prec of the inner operator and vectors */
    int inner_recon;   /* 18 or 12: links of the inner operator */
    int outer_recon;   /* 18 or 12: links of the reliable updates' operator */
    int reliable;      /* 1 reliable updates, 0 iterative refinement */
    double delta;      /* see above; ignored for inner_prec = WD_F64 */
    int maxiter;       /* limit on inner iterations */
    int autotune;      /* 1: tune the hop launches the solve uses (once per context) */
    int use_graph;     /* 1 (mixed precision, reliable = 1): a CUDA graph whose device-side
                          loop runs iterations (CG scalars on the device) until a reliable
                          update is due, or 32 of them; the host does the FP64 updates
                          between launches */
    int outer_prec;    /* WD_F64 (0) or WD_DF: arithmetic of the operator that recomputes
                          the true residual at a reliable update (mixed precision only;
                          ignored for inner_prec = WD_F64).  x, b, the residual and all
                          inner products stay FP64.  WD_DF applies A in double-word FP32
                          (errors of order 2^-48 |A| |x|), about 3 times faster than FP64
                          on a part whose FP64 rate is 1/64 of its FP32 rate.  Updates
                          that check convergence (the iterated residual has met the
                          target), a double-word residual that meets it, and all updates
                          after a failed check use the FP64 operator, so only an FP64
                          residual ends the solve (and is reported): convergence means
                          the same with either setting. */
} wd_cg_opts;

typedef struct {
    int iters;             /* inner iterations */
    int reliable_updates;  /* true-residual recomputations (FP64 or double-word) */
    int status;            /* wd_status of the solve */
    double true_rel_resid; /* final |b - A x| / |b|, FP64 */
    double seconds;        /* host wall time of the call */
} wd_cg_stats;

int cg_solve(wd_ctx *ctx, const wd_gauge *g, double mass, void *x_e, const void *b_e, double tol,
             const wd_cg_opts *opts, wd_cg_stats *stats, void *stream);

/* ---- BiCGStab on Mhat and the full-system solve -----------------------------
 * The paper names only CG (Sec. II-A); these are the steps either side of the
 * CG path.
 *
 * bicgstab_solve: Mhat x_e = b_e on the even sites (Mhat as for cg_solve, not
 * Hermitian) by BiCGStab (van der Vorst 1992), x_0 = 0, shadow residual b_e.
 * x_e, b_e: even half fields in WD_F64 (device).  Converged when the FP64 true
 * residual |b - Mhat x| / |b| <= tol.  Options as for cg_solve: inner_prec =
 * WD_F64 plain FP64; otherwise the iterated vectors and operator use
 * inner_prec storage with FP32 arithmetic, the solution, the true residual and
 * all inner products FP64, and reliable = 1 replaces the iterated residual by
 * the true one (FP64 operator) when it has dropped by `delta` since the last
 * replacement (the Krylov state is kept), reliable = 0 restarts BiCGStab on the
 * true residual each time (iterative refinement).  A breakdown (zero <r^, v>,
 * omega or rho) restarts from the true residual.  use_graph is ignored.
 * stats->iters counts BiCGStab iterations (two Mhat applications each).
 *
 * wilson_solve: D x = b on the full lattice, D = (m+4) - H/2.  x, b: full
 * fields in WD_F64 (even half, then odd half; device).  Even-odd reduction:
 * b^_e = b_e + H_eo b_o / (2(m+4)), solve Mhat x_e = b^_e to the relative
 * residual tol |b| / |b^_e| (the even rows of D x = b then leave exactly that
 * residual), then x_o = (b_o + H_oe x_e / 2) / (m+4), which satisfies the odd
 * rows.  solver = WD_SOLVER_BICGSTAB: the Schur system by BiCGStab as above;
 * WD_SOLVER_CGNE: by CG on Mhat^dagger Mhat x_e = Mhat^dagger b^_e (all
 * cg_solve options, use_graph included), repeated on the Schur residual until
 * it is small enough.  stats->true_rel_resid = |b - D x| / |b| with the FP64
 * operator; WD_ENOCONV if it is above tol.
 *
 * Both: synchronous; workspace owned by the context; x must not alias b. */
typedef enum { WD_SOLVER_CGNE = 0, WD_SOLVER_BICGSTAB = 1 } wd_solver;

int bicgstab_solve(wd_ctx *ctx, const wd_gauge *g, double mass, void *x_e, const void *b_e, double tol,
                   const wd_cg_opts *opts, wd_cg_stats *stats, void *stream);
int wilson_solve(wd_ctx *ctx, const wd_gauge *g, double mass, void *x, const void *b, double tol, int solver,
                 const wd_cg_opts *opts, wd_cg_stats *stats, void *stream);

/* ---- Batches of solves (different lattices, masses, tolerances) --------------
 * Each descriptor is one cg_solve problem; its lattice comes from its gauge.
 * Modes:
 *   WD_BATCH_SEQUENTIAL  cg_solve on each descriptor in turn (any options);
 *   WD_BATCH_GRAPH       mixed-precision reliable-update solves (inner_prec
 *                        WD_F32/WD_F16/WD_BF16) run as the request groups of
 *                        the serving queue (rq_*): the solves of one gauge,
 *                        inner precision and inner link format iterate in one
 *                        CUDA graph with a device-side loop and one
 *                        shared-link launch per hop for all of them; FP64
 *                        reliable updates on each solve's own stream, the
 *                        convergence test on the host between launches;
 *   WD_BATCH_PERSISTENT  one cooperative kernel: each solve runs on its own
 *                        group of thread blocks (sized by volume), steps
 *                        separated by group barriers whose waits are bounded
 *                        (1 s of clock cycles; WD_BARRIER_TIMEOUT_S overrides);
 *                        options must be inner_prec WD_F32, WD_F16 or WD_BF16
 *                        (the same for all), 18-real links, reliable = 1.
 *                        Batches larger than one co-resident grid run as
 *                        several launches.
 * stats[k] receives solve k's statistics; `seconds` is the wall time of the
 * whole call.  Returns the first failure (WD_ENOCONV, WD_ETIMEOUT, ...).
 * Synchronous; allocates its workspace for the duration of the call. */
typedef enum { WD_BATCH_SEQUENTIAL = 0, WD_BATCH_GRAPH = 1, WD_BATCH_PERSISTENT = 2 } wd_batch_mode;

typedef struct {
    const wd_gauge *gauge;
    double mass;
    double tol;
    void *x_e;          /* even half field, WD_F64, device (output) */
    const void *b_e;    /* even half field, WD_F64, device */
    wd_cg_opts opts;
} wd_solve_desc;

int cg_solve_batch(wd_ctx *ctx, int n, const wd_solve_desc *descs, int mode, wd_cg_stats *stats,
                   void *stream);

/* ---- Request queue with continuous batching (serving) ------------------------
 * rq_create starts a scheduler thread for the context's device.  Requests are
 * wd_solve_desc problems (mixed-precision reliable-update CG: inner_prec
 * WD_F32, WD_F16 or WD_BF16) whose gauge and fields stay resident; x_e and b_e
 * are the caller's device buffers and must stay valid until the request's
 * result has been taken.  The scheduler admits waiting requests while fewer
 * than max_slots run and their workspace fits hbm_budget_bytes (first come
 * first served, a request that fits may pass one that does not).  Each
 * admitted request has its own workspace and stream and joins the request
 * group of its gauge, inner precision and inner link format (up to 32
 * members; another group opens when one is full).  A group runs the
 * low-precision CG iterations of its ready members together in a graph whose
 * device-side loop launches each of the four even-odd hops once for all of
 * them, with the links of each block's sites loaded once and applied to every
 * member's field (each member with its own mass, tolerance and scalars), and
 * stops when any member needs its FP64 reliable update or after 16
 * iterations.  The scheduler then enqueues those updates on the members' own
 * streams, relaunches the group with the others, and lets members join or
 * rejoin (after their update) at the next launch.  A member's results do not
 * depend on the other members: alone and in any mix it gets the same bits.
 * Groups of different gauges and the updates run concurrently on their own
 * streams.
 *   rq_submit: non-blocking, thread-safe; copies the descriptor; WD_ENOMEM if
 *              the request alone exceeds the budget.
 *   rq_poll:   WD_EBUSY while running; otherwise fills the result and forgets
 *              the ticket.
 *   rq_wait:   blocks up to timeout_ms (< 0: forever); WD_ETIMEOUT if still
 *              running (the request keeps running).
 *   rq_cancel: a waiting request ends at once with WD_ECANCELLED; a running one
 *              when its current launch or reliable update has finished.
 *   rq_destroy: finishes every submitted request, then stops and frees.
 * Times in wd_solve_result are seconds since rq_create.  A request whose
 * source is not finite ends with WD_EINVAL without affecting the others. */
typedef struct rq_queue rq_queue;

typedef struct {
    int status;          /* wd_status of the solve */
    wd_cg_stats stats;   /* stats.seconds = t_finish - t_submit */
    double t_submit, t_admit, t_start, t_finish;
} wd_solve_result;

typedef struct {
    uint64_t submitted, completed, admission_stalls, steps;   /* steps: group launches + reliable updates */
    double mean_running;     /* running requests, averaged over the time any request runs */
    int waiting, running;
    size_t hbm_in_use;
    uint64_t group_launches; /* launches of group loops (each one shared by its members) */
    double mean_group_size;  /* members per group launch, averaged over the launches */
} rq_counters;

/* Device workspace bytes one queued (or graph-batched) solve on this lattice
 * allocates while it runs: what the queue counts against its budget. */
int wd_solve_workspace_bytes(const int dims[4], int inner_prec, size_t *out);

int rq_create(wd_ctx *ctx, size_t hbm_budget_bytes, int max_slots, rq_queue **out);
int rq_submit(rq_queue *q, const wd_solve_desc *desc, uint64_t *ticket);
int rq_poll(rq_queue *q, uint64_t ticket, wd_solve_result *out);
int rq_wait(rq_queue *q, uint64_t ticket, int timeout_ms, wd_solve_result *out);
int rq_cancel(rq_queue *q, uint64_t ticket);
int rq_stats(rq_queue *q, rq_counters *out);
int rq_destroy(rq_queue *q);

#ifdef __cplusplus
}
#endif
#endif /* WDIRAC_H */
