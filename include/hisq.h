/*
 * hisq.h - C ABI of the GB300 multi-right-hand-side HISQ Dslash and CG library.
 *
 * The operator is the HISQ staggered Dslash of Kaczmarek, Schmidt,
 * Steinbrecher and Wagner, "Conjugate gradient solvers on Intel Xeon Phi and
 * NVIDIA GPUs" (GPUHEP2014), Eq. 3, applied to a bundle of n right-hand
 * sides at once as in Eq. 4:
 *
 *   w(x) = sum_{mu=0..3} [ U_mu(x) v(x+mu) - U_mu(x-mu)^dag v(x-mu)
 *                         + N_mu(x) v(x+3mu) - N_mu(x-3mu)^dag v(x-3mu) ]
 *
 * and the conjugate-gradient inversion of the fermion matrix M = 2m + D that
 * takes most of the runtime of the stochastic trace estimates of Eq. 2.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice L[4] = {Lx, Ly, Lz, Lt}; every extent even and >= 4.
 * Directions mu = 0,1,2,3 are x,y,z,t. V = Lx*Ly*Lz*Lt, V_h = V/2.
 * Lexicographic site index i = x + Lx*(y + Ly*(z + Lz*t)).
 * Parity p = (x+y+z+t) % 2. Half-lattice index h = i/2 enumerates the V_h
 * sites of one parity in lexicographic order.
 *
 * Canonical links: complex128 [4][V][3][3] (mu-major, lexicographic site,
 * row-major colour, interleaved re/im). U[mu][i] is the link from site i to
 * i+mu, N[mu][i] the link from i to i+3mu. Staggered phases, boundary signs
 * and the Naik coefficient are folded into the links by the caller.
 *
 * Spinors (colour vectors) of one parity: [V_h][3] complex, interleaved re/im,
 * element type by hisq_prec (F64: double, F32: float, F16: IEEE half).
 * Full-lattice vectors (only for mu != 0 solves) are parity-blocked:
 * [2][V_h][3], the V_h even sites first.
 *
 * Ownership: the library owns every hisq_gauge and the workspaces cached on
 * it (device memory it allocates with cudaMalloc and frees in
 * hisq_gauge_free). The caller owns every spinor buffer; pointers are
 * borrowed for the duration of the call, stream-ordered on `stream`
 * (a cudaStream_t; NULL = legacy default stream).
 *
 * Errors: every call returns a hisq_status; nothing aborts or throws across
 * the ABI. hisq_last_error() returns a thread-local message for the last
 * failing call on this thread.
 *
 * Thread safety: calls on different handles are independent. Calls that
 * share a handle must be serialised by the caller (they share workspaces).
 */
#ifndef HISQ_H
#define HISQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int hisq_status;
enum {
    HISQ_OK = 0,
    HISQ_EINVAL = 1,      /* bad argument: extents, n, pointer, alignment, mode */
    HISQ_ERECON = 2,      /* links not representable in the requested compression */
    HISQ_ENOCONV = 3,     /* CG hit maxiter before every rhs converged */
    HISQ_EBREAKDOWN = 4,  /* CG breakdown: <p,Ap> <= 0 or not finite */
    HISQ_ENAN = 5,        /* non-finite value in a source or residual */
    HISQ_ECUDA = 6,       /* a CUDA runtime call failed; see hisq_last_error() */
    HISQ_ETIMEOUT = 7,    /* a bounded device-side wait gave up (staged-link kernel) */
    HISQ_ENOMEM = 8       /* device allocation failed */
};

typedef int hisq_prec;
enum { HISQ_F64 = 0, HISQ_F32 = 1, HISQ_F16 = 2 };

typedef int hisq_recon;
enum { HISQ_R18 = 18, HISQ_R12 = 12, HISQ_R14 = 14 };

/* Spinor layout on one parity: AoS [V_h][3] per rhs (colour fastest), SoA
 * [3][V_h] per rhs (site fastest, one plane per colour), or the bundle layout
 * of all n rhs together in one buffer (FP32 and FP16 storage only): 16-byte
 * chunks, each one colour of W consecutive rhs at one site with the W real
 * parts first and then the W imaginary parts (W = 2 for FP32: float
 * re_k, re_k+1, im_k, im_k+1; W = 4 for FP16: 4 halves of real parts, 4 of
 * imaginary parts), chunk (g = k / W, colour c, site h) at index
 * (3 g + c) V_h + h. n must be a multiple of W. A warp of 32 neighbouring
 * sites then reads whole 512-byte rows for every hop of Eq. 3, and a link
 * load serves W rhs per chunk. */
typedef int hisq_layout;
enum { HISQ_AOS = 0, HISQ_SOA = 1, HISQ_BUNDLE = 2 };

typedef struct hisq_gauge_s* hisq_gauge;

/* Library version, major*10000 + minor*100 + patch. */
int hisq_version(void);

/* Message describing the last failing call on this thread ("" if none). */
const char* hisq_last_error(void);

/*
 * Link compression, Sec. 1: the paper stores symmetric links in fewer reals
 * and notes that for the HISQ action only the Naik links keep enough
 * structure for it (9 or 13/14 reals). Encodings built here:
 *   R18: all 9 complex entries.
 *   R14: rows 1 and 2 plus one complex z; row 3 = z * conj(row1 x row2).
 *        Exact for any link c*W, c real, W unitary (z = det(W)/c). Valid for
 *        fat and Naik links.
 *   R12: rows 1 and 2; row 3 = (sigma/s) * conj(row1 x row2) with sigma the
 *        staggered sign eta_mu(x) * bc(x,mu) recomputed from coordinates
 *        (antiperiodic t) and s = |row 1| of U[0][0]. Exact only for links
 *        s * sigma * SU(3); fat links only (recon_N may not be R12).
 *
 * hisq_gauge_load packs U and N into the internal site-major SoA layout
 * [parity][mu][complex component][V_h] in precision `prec`, and always also
 * keeps an FP64 R18 copy used by FP64 Dslash calls and by the CG's FP64
 * reliable updates. prec == HISQ_F64 requires R18 for both fields.
 * prec == HISQ_F16 stores every link real as a 16-bit integer q with value
 * q * s_c, one scale s_c = max |Re|,|Im| / 32767 per stored complex
 * component c of each field (2^-15 of the range, where IEEE half keeps only
 * 2^-11 of each value: with IEEE half links the sloppy operator differs from
 * the FP64 one by more than its smallest eigenvalue at light masses and the
 * reliable-update CG diverges); FP16 spinors stay IEEE half.
 *   L          lattice extents (host array of 4 ints).
 *   U, N       canonical complex128 links, device pointers if on_device != 0,
 *              else host pointers. Read only; not retained.
 *   recon_tol  largest allowed |reconstructed - input| entry (FP64, before
 *              rounding to `prec`); exceeding it returns HISQ_ERECON and
 *              no handle.
 *   out        receives the new handle on HISQ_OK.
 * Synchronises `stream` before returning.
 */
hisq_status hisq_gauge_load(const int L[4], const void* U, const void* N,
                            int on_device, hisq_prec prec, hisq_recon recon_U,
                            hisq_recon recon_N, double recon_tol, void* stream,
                            hisq_gauge* out);

/* Frees the handle, its link copies and every cached workspace. NULL is a no-op. */
hisq_status hisq_gauge_free(hisq_gauge g);

/* Storage precision and reconstruct modes of a handle (any pointer may be NULL). */
hisq_status hisq_gauge_info(hisq_gauge g, int L[4], hisq_prec* prec,
                            hisq_recon* recon_U, hisq_recon* recon_N,
                            size_t* device_bytes);

/*
 * Tuning of the Dslash thread mapping for this handle: rhs handled per
 * thread (1, 2, 4, 8; FP64: 1, 2, 4) and the minimum resident blocks per SM
 * the kernel is compiled for (register budget); 0 = automatic. Flags:
 * HISQ_MAP_PACKED for paired FP32 (f32x2) complex arithmetic,
 * HISQ_MAP_L2_PREFETCH to bulk-prefetch each tile's links into L2,
 * HISQ_MAP_STAGED to stage each tile's links in shared memory with bulk
 * asynchronous copies (FP32/FP16 storage; tiles of 128 sites made of whole
 * x-rows inside one y-z plane, at most 2 rhs groups), HISQ_MAP_PIPELINED /
 * HISQ_MAP_PIPELINED2 to keep the link and neighbour loads of the next one /
 * two hops in flight while the current hop is multiplied (FP32/FP16). At
 * most one of PACKED, STAGED, PIPELINED, PIPELINED2. Mappings that are not
 * built or do not fit n or the lattice fall back to the automatic choice.
 */
enum {
    HISQ_MAP_PACKED = 1,
    HISQ_MAP_L2_PREFETCH = 2,
    HISQ_MAP_STAGED = 4,
    HISQ_MAP_PIPELINED = 8,
    HISQ_MAP_PIPELINED2 = 16,
    HISQ_MAP_COMPACT = 128,
    HISQ_MAP_TILE_XY = 256
};
/* On the bundle layout (rhs per thread 4 or 8, min blocks per SM of 128-thread
 * blocks 1..4) the kernel multiplies rhs pairs with packed FP32 (f32x2)
 * instructions and keeps the next hop's link load in flight; flags select
 * variants: HISQ_MAP_PIPELINED also the next hop's neighbour chunks,
 * HISQ_MAP_COMPACT a hop loop with the direction as a runtime loop (a quarter
 * of the code, one colour of the neighbours converted at a time),
 * HISQ_MAP_STAGED the neighbour chunks copied into shared memory by
 * asynchronous per-thread copies one hop ahead (two with HISQ_MAP_PIPELINED2;
 * together with HISQ_MAP_COMPACT one, or three with HISQ_MAP_PIPELINED2).
 * HISQ_MAP_TILE_XY the neighbours of the x and y hops read from a
 * shared-memory tile of whole x-rows of the block's (z, t) plane (loaded while
 * the z and t hops run; one rhs group, i.e. n equal to rhs per thread, and
 * planes of whole 128-site runs, else the plain loop).
 * Defaults at 8 rhs per thread: FP16 storage STAGED | COMPACT at 4 blocks per
 * SM, FP32 storage no flag at 3 blocks per SM. */
hisq_status hisq_set_dslash_mapping(hisq_gauge g, int rhs_per_thread, int min_blocks,
                                    int flags);

/* The mapping a Dslash of n rhs in `spinor_prec` will use on this handle:
 * rhs per thread, min blocks per SM and HISQ_MAP_* flags (host pointers), for
 * the AoS layout (hisq_get_dslash_mapping) or a given layout (_ex; the bundle
 * layout returns HISQ_EINVAL when n does not fit it). */
hisq_status hisq_get_dslash_mapping(hisq_gauge g, int n, hisq_prec spinor_prec,
                                    int* rhs_per_thread, int* min_blocks, int* flags);
hisq_status hisq_get_dslash_mapping_ex(hisq_gauge g, int n, hisq_prec spinor_prec,
                                       hisq_layout layout, int* rhs_per_thread,
                                       int* min_blocks, int* flags);

/*
 * Autotuner: times `reps` Dslash launches of every built mapping that fits
 * n rhs, `spinor_prec` and `layout` on this handle (register, pipelined and
 * shared-memory-staged kernels, every register budget) and keeps the fastest for
 * later calls of that shape (hisq_set_dslash_mapping still takes priority).
 * Returns the choice and its time per launch (any output may be NULL).
 * Allocates and frees scratch spinors; synchronises the device.
 */
hisq_status hisq_autotune_dslash(hisq_gauge g, int n, hisq_prec spinor_prec,
                                 hisq_layout layout, int reps, int* rhs_per_thread,
                                 int* min_blocks, int* flags, double* seconds);

/*
 * Gauge load with an autotuned link compression (the paper compares the
 * 18-real and 14-real Naik storage in Table 1 and Sec. 1; 12 reals for the
 * fat links where exact): loads the links, exactly as hisq_gauge_load, with
 * every (recon_U, recon_N) pair that has a kernel for `prec` (F64: 18/18;
 * F32/F16: 18/18, 18/14, 12/14, 14/14), skips pairs that do not hold the
 * links within recon_tol, runs hisq_autotune_dslash for n rhs in every spinor
 * layout that fits n on each, and returns in *out the handle whose Dslash in
 * the CG's layout (the bundle layout where n fits it, else AoS) was fastest,
 * with its tuned mappings. hisq_gauge_info reports the
 * chosen compression. The choice is cached per (L, n, prec) for the life of
 * the process; later calls load that pair directly (and search again if it
 * does not hold their links). Transient device memory:
 * two handles. Errors as hisq_gauge_load; HISQ_ERECON if no pair holds.
 */
hisq_status hisq_gauge_load_tuned(const int L[4], const void* U, const void* N, int on_device,
                                  hisq_prec prec, int n, double recon_tol, void* stream,
                                  hisq_gauge* out);

/*
 * Bundle-size search (Eq. 4 shares each link load among the n rhs of a
 * bundle; Table 1 gives the arithmetic intensity as a function of n): times
 * the autotuned Dslash for n = 1, 2, 4, ... <= n_max (n_max <= 16) and returns
 * the bundle size with the lowest seconds per rhs and that time. The tuned
 * mapping of every size tried stays cached on the handle.
 */
hisq_status hisq_autotune_bundle(hisq_gauge g, int n_max, hisq_prec prec, hisq_layout layout,
                                 int reps, int* best_n, double* seconds_per_rhs);

/*
 * Compress a canonical link field to `r` reals per link (R18/R14/R12, same
 * encodings as above) and back. Both take device pointers.
 *   links   complex128 [4][V][3][3]
 *   packed  double [4][V][r]
 * hisq_link_compress also writes the largest reconstruction error to
 * *max_err (host pointer, may be NULL). Synchronises `stream`.
 */
hisq_status hisq_link_compress(const int L[4], const void* links, hisq_recon r,
                               void* packed, double* max_err, void* stream);
hisq_status hisq_link_reconstruct(const int L[4], const void* packed,
                                  hisq_recon r, void* links, void* stream);

/*
 * Multi-rhs Dslash, Eq. 3 and Eq. 4: w[k] = D_{p,1-p} v[k] for k < n, i.e. the
 * output sites have parity `parity` and the inputs the opposite parity (every
 * one- and three-hop flips parity). One launch reads every link once for all
 * n right-hand sides.
 *   v, w         host arrays of n device pointers, each [V_h][3] complex of
 *                `spinor_prec`; w[k] must not alias any v[j].
 *   n            1..16.
 *   spinor_prec  F64 uses the FP64 R18 links; F32 and F16 use the handle's
 *                storage copy, which must then have that same precision.
 * hisq_dslash uses the AoS layout. hisq_dslash_ex takes the spinor layout and
 * adds a chemical potential mu on the temporal hops: forward one-hop
 * x e^{+mu}, backward one-hop x e^{-mu}, forward Naik x e^{+3mu}, backward
 * Naik x e^{-3mu}. With layout HISQ_BUNDLE, v and w hold one pointer each,
 * the bundle buffers of all n rhs (n a multiple of the chunk width W; F32 or
 * F16 only; 16-byte aligned). Asynchronous on `stream`.
 */
hisq_status hisq_dslash(hisq_gauge g, const void* const v[], void* const w[],
                        int n, int parity, hisq_prec spinor_prec, void* stream);
hisq_status hisq_dslash_ex(hisq_gauge g, double mu, const void* const v[],
                           void* const w[], int n, int parity,
                           hisq_prec spinor_prec, hisq_layout layout,
                           void* stream);

/*
 * Conversion between n FP64 vectors and one bundle (layout HISQ_BUNDLE, see
 * hisq_layout) of storage precision F32 or F16, for the bundle Dslash and the
 * CG. src / dst: host arrays of n device pointers to complex128 [V_h][3] on
 * one parity (V_h = V / 2 of the handle's lattice); bundle: device pointer to
 * n * 3 * V_h complex numbers of `prec` (16-byte aligned). Packing rounds to
 * `prec` (round to nearest). n must be a multiple of W (2 for F32, 4 for
 * F16), at most 16. The paper's layouts are per-rhs arrays; this interleave
 * is this library's (Sec. 2 notes a per-site rhs-contiguous layout helped on
 * Xeon Phi). Asynchronous on `stream`.
 */
hisq_status hisq_bundle_pack(hisq_gauge g, const void* const src[], int n, hisq_prec prec,
                             void* bundle, void* stream);
hisq_status hisq_bundle_unpack(hisq_gauge g, const void* bundle, int n, hisq_prec prec,
                               void* const dst[], void* stream);

/*
 * Even-odd normal operator of M = 2m + D at mu = 0 (Sec. 1: the fermion
 * matrix is inverted; its hopping part is the Dslash of Eq. 3, which only
 * couples opposite parities, so M^dag M splits into parity blocks):
 *   w[k] = A_e v[k] = 4 m^2 v[k] - D_eo D_oe v[k]   (even sites)
 * A_e = (M^dag M) restricted to even sites, Hermitian positive definite.
 * v, w as for hisq_dslash with parity 0. Uses a cached odd-parity temporary on
 * the handle. Asynchronous on `stream`.
 */
hisq_status hisq_mdagm(hisq_gauge g, double mass, const void* const v[],
                       void* const w[], int n, hisq_prec spinor_prec,
                       void* stream);

/*
 * Full-lattice fermion matrix M(mu) = 2m + D(mu) and its relatives on
 * parity-blocked vectors [2][V_h][3] (even half first):
 *   HISQ_OP_M      w = M(mu) v
 *   HISQ_OP_MDAG   w = M(mu)^dag v = 2m v - D(-mu) v
 *   HISQ_OP_DM_DMU w = dM/dmu v: the temporal hops only, with factors
 *                  +e^{mu}, +e^{-mu} (one-hop) and +3e^{3mu}, +3e^{-3mu} (Naik)
 *                  on U v(x+t), U^dag v(x-t), N v(x+3t), N^dag v(x-3t).
 * M(mu) is the matrix whose mu-derivatives enter the stochastic traces of
 * Eq. 2. v and w: n device pointers each; w must not overlap any v.
 * Asynchronous on `stream`.
 */
enum {
    HISQ_OP_M = 0,
    HISQ_OP_MDAG = 1,
    HISQ_OP_DM_DMU = 2,    /* k-th derivative: HISQ_OP_DM_DMU + k - 1, k = 1..4; */
    HISQ_OP_D2M_DMU2 = 3,  /* the factors become +e^{mu}, +(-1)^k e^{-mu} on    */
    HISQ_OP_D3M_DMU3 = 4,  /* the one-hops and 3^k e^{3mu}, (-3)^k e^{-3mu} on  */
    HISQ_OP_D4M_DMU4 = 5   /* the Naik hops (signs as for the first derivative) */
};
hisq_status hisq_apply_m(hisq_gauge g, double mass, double mu, int op,
                         const void* const v[], void* const w[], int n,
                         hisq_prec spinor_prec, void* stream);

/*
 * Link force for gradients of a solve (derivatives of the stochastic trace
 * estimators of Eq. 2, Sec. 1, with respect to the links of Eq. 3). For
 * FP64 parity-blocked vectors a_k,
 * b_k ([2][V_h][3] complex128, device) accumulates into `out` (device,
 * complex128 [4][V][3][3], canonical link layout)
 *   out[mu][x] += coef * sum_k [ f a_k(x) b_k(x+hop mu)^dag
 *                               - (1/f) b_k(x) a_k(x+hop mu)^dag ]
 * with f = e^{hop mu} on temporal links (1 otherwise); hop = 1 for the fat
 * links U, 3 for the Naik links N. This is the derivative (d/dRe + i d/dIm)
 * of Re sum_k a_k^dag D(mu) b_k with respect to each link. Asynchronous.
 */
hisq_status hisq_link_force(hisq_gauge g, double mu, int hop, const void* const a[],
                            const void* const b[], int n, double coef, void* out,
                            void* stream);

/*
 * The bilinears eta^dag X eta of Eq. 2 (Sec. 1), per rhs:
 * out[2k] + i out[2k+1] = <a_k, b_k> = sum_i conj(a_k[i]) b_k[i] over `len`
 * complex128 numbers, in FP64 with a fixed summation order. a, b: n device
 * pointers; out: host array of 2n doubles. Uses reduction scratch owned by
 * the handle. Synchronises `stream`.
 */
hisq_status hisq_cdot(hisq_gauge g, const void* const a[], const void* const b[], int n,
                      long long len, double* out, void* stream);

/*
 * hisq_cdot without any device allocation. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc, such as
 * processes whose device memory is entirely owned by another allocator (an
 * extra allocation would fail or fragment its pool) and latency-critical
 * code that cannot accept the device synchronisation cudaMalloc implies.
 * Same operation, arguments and result as hisq_cdot, without a handle: the
 * reduction scratch is a fixed device array of about 1 MiB inside the
 * library, which every GPU that loads the library holds until the process
 * exits. n is limited to 16, the bundle size that array holds; larger n
 * returns HISQ_EINVAL.
 *   - The first call on a device looks up the array's device address there
 *     (cudaGetSymbolAddress with that device current); make that first call
 *     before starting any stream capture.
 *   - Every call on a device shares the one array and leaves its last
 *     contents there; each call clears the part that must start at zero.
 *     Calls whose kernels overlap on the GPU (other streams, other host
 *     threads) race on the array: serialise them.
 * Synchronises `stream`.
 */
hisq_status hisq_cdot_noalloc(const void* const a[], const void* const b[], int n,
                              long long len, double* out, void* stream);

/* CG parameters; hisq_cg_default_params fills the defaults noted below. */
typedef struct {
    int maxiter;           /* iteration cap (100000) */
    int reliable_every;    /* FP64 reliable update every K iterations (50) */
    double reliable_delta; /* ... or when ||r|| drops by this factor (0.1) */
    hisq_prec inner_prec;  /* storage precision of the inner iteration (F32) */
    int use_x0;            /* 1: x holds an initial guess on entry (0) */
    int even_odd;          /* 1: even-odd system at mu = 0 (1) */
    int check_every;       /* iterations between convergence / reliable-update decisions (10) */
    int use_graphs;        /* 1: replay iterations from a captured CUDA graph (1) */
    int rhs_per_thread;    /* Dslash rhs per thread: 0 = auto, else 1/2/4/8 */
    hisq_layout spinor_layout; /* layout of the CG's internal low-precision vectors
                                  (HISQ_BUNDLE; where n is not a multiple of the
                                  chunk width, or for F64 and full-lattice solves,
                                  the solve uses HISQ_AOS) */
    int device_loop;       /* 1: the whole solve is one graph launch whose
                              conditional nodes take every decision on the
                              device (needs use_graphs, and maxiter and
                              reliable_every multiples of check_every; else
                              the host decides after every check_every
                              iterations) (1) */
    int profile_kernels;   /* 1: time the four launches of every iteration
                              with CUDA events on the solve's stream and
                              report their mean durations in
                              hisq_cg_stats.kernel_us; the solve then launches
                              every kernel from the host (no graphs, no device
                              loop), which costs launch overhead (0) */
} hisq_cg_params;

typedef struct {
    int iters[16];             /* iterations until each rhs converged */
    int total_iters;           /* iterations of the bundle */
    int reliable_updates;      /* FP64 residual recomputations */
    double true_rel_res[16];   /* final ||b - A x|| / ||b|| in FP64 per rhs */
    double seconds;            /* wall time of the solve, host clock */
    int profiled_iters;        /* iterations timed by profile_kernels (0 if off) */
    double kernel_us[4];       /* with profile_kernels: mean device time (us) per
                                  iteration of [0] t = D_oe p (both Dslash of the
                                  full-lattice operator y = M p), [1] Ap and the
                                  reduction forming alpha, [2] r -= alpha Ap with
                                  |r|^2 and beta, [3] x += alpha p, p = r + beta p */
} hisq_cg_stats;

void hisq_cg_default_params(hisq_cg_params* p);

/*
 * The inversion of the fermion matrix for many random vectors at once
 * (abstract; Sec. 1: the vectors of a bundle share each Dslash of Eq. 4;
 * Sec. 3: the CG with several rhs). Independent coefficients per vector
 * (no block Krylov space) are this library's reading. Conjugate gradient on the normal
 * equations of M = 2m + D, n independent
 * CGs (one per rhs, own alpha and beta) sharing every Dslash. Stops rhs k
 * when ||b_k - A x_k|| / ||b_k|| <= tol in FP64 (tol > 0). p may be NULL
 * (defaults); stats may be NULL.
 *   even_odd = 1 (requires mu == 0): (4m^2 - D_eo D_oe) x_e = b_e, b and x
 *       [V_h][3] complex128 on even sites.
 *   even_odd = 0: M(mu)^dag M(mu) x = b on the full lattice, with
 *       M(mu)^dag = 2m - D(-mu); b and x parity-blocked [2][V_h][3].
 * b[k], x[k] are device or host pointers (detected per pointer); host data
 * is copied in and out on `stream`. The inner iteration stores vectors in
 * p->inner_prec with FP32 arithmetic (FP64 if inner_prec is F64); every
 * reliable update recomputes r = b - A x in FP64 with FP64 links and adds
 * the low-precision solution increment into the FP64 x. Convergence is
 * declared per rhs on the FP64 true residual only.
 * Returns HISQ_OK when every rhs reached p->tol, HISQ_ENOCONV at maxiter,
 * HISQ_EBREAKDOWN, HISQ_ENAN (after any of these three, x[k] holds the
 * solution at the lowest FP64 residual rhs k reached, which is the residual
 * stats->true_rel_res reports), HISQ_EINVAL (bad n, tol, pointers or mu != 0
 * with even_odd).
 * Synchronises `stream` before returning.
 */
hisq_status hisq_cg_solve(hisq_gauge g, double mass, double mu,
                          const void* const b[], void* const x[], int n,
                          double tol, const hisq_cg_params* p,
                          hisq_cg_stats* stats, void* stream);

/*
 * Several independent solves advanced together (Sec. 3, Fig. 4 right: the
 * inverter for a fixed number of rhs on lattices of different size), e.g.
 * bundles on gauge fields
 * of uneven volume: each chunk of iterations of all unfinished solves is one
 * CUDA graph whose branches run the solves concurrently, so small lattices
 * share the GPU instead of running one after another. Every problem has its
 * own handle (distinct handles required), mass, mu, bundle, size and
 * tolerance, with the meaning of hisq_cg_solve; the parameters p are shared.
 * stats (may be NULL) receives one entry per problem. Returns HISQ_OK when
 * every problem converged, else the first failing problem's status.
 */
typedef struct {
    hisq_gauge g;
    double mass;
    double mu;
    const void* const* b;
    void* const* x;
    int n;
    double tol;
} hisq_cg_problem;

hisq_status hisq_cg_solve_batched(const hisq_cg_problem* problems, int nprob,
                                  const hisq_cg_params* p, hisq_cg_stats* stats,
                                  void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HISQ_H */
