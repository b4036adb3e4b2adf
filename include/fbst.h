/*
 * fbst.h -- C ABI of the GB300 (sm_103a) fast broadband beamspace transform (FBST).
 *
 * The FBST (Singh, DeLude, Davenport, Romberg, "A Fast Broadband Beamspace Transformation")
 * forms B broadband beams from N snapshots of an M-element array. For each beam b it computes
 * the regularised least-squares beam of Sec. III-A,
 *
 *     w_b    = F_b^H y                          Eq. (5)-(6); the "fan" chirp-z of Sec. IV
 *     beta_b = (F_b^H F_b + delta I)^{-1} w_b   Eq. (5); Toeplitz, applied as in Sec. V
 *     bhat_b = F_u beta_b                       Eq. (7); a chirp-z in n (Sec. V)
 *
 * Conventions shared by every entry point (all 0-based, time in samples):
 *   - complex numbers are complex64: interleaved (re, im) float32 pairs, 8 bytes each;
 *   - y    is [nblk][M][N]: block, element, snapshot (snapshot fastest);
 *   - w    is [nblk][B][L]: block, beam, frequency index (frequency fastest);
 *   - bhat is [nblk][B][N]: block, beam, output sample;
 *   - element m of a linear array sits at m half wavelengths (at f_c + Omega) from element 0;
 *     element s = kx*my + ky of a rectangular array sits at (kx, ky);
 *   - beam b of a linear array looks at u_b = -1 + 2b/B (direction cosine); beam b = a*by + c of a
 *     rectangular array looks at (u, v) = (-1 + 2a/bx, -1 + 2c/by) (Sec. IV, App. B);
 *   - frequency index ell = 0..L-1 stands for the paper's ell = 1..L, ell' = ell + 1 - L/2, and
 *     omega_ell*T_s = 2*pi*epsilon*ell'/L (Eq. (3)).
 *
 * Device pointers must be 16-byte aligned and must not overlap. Every entry point returns an
 * fbst_status; nothing crosses the ABI as an exception. Execution entry points enqueue work on
 * the given CUDA stream (a cudaStream_t passed as void*, NULL = legacy default stream) and return
 * before it finishes; results are valid once the stream is synchronised. Plans are not
 * thread-safe: calls that share a plan must not run concurrently from several host threads, and
 * executions of one plan on different streams must not overlap in time on the GPU (they share
 * the plan's workspace).
 */
#ifndef FBST_H
#define FBST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fbst_plan_s* fbst_plan_t;

/* Status codes returned by every entry point. */
enum fbst_status {
  FBST_OK = 0,
  FBST_ERR_INVALID = -1,     /* a size, pointer or parameter is out of range */
  FBST_ERR_OOM = -2,         /* device or host allocation failed */
  FBST_ERR_CUDA = -3,        /* a CUDA runtime call or kernel launch failed */
  FBST_ERR_UNSUPPORTED = -4, /* valid but not implemented (e.g. an FFT size above 4096) */
  FBST_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
  FBST_ERR_NUMERIC = -6      /* plan-time maths failed (A_b not numerically positive definite) */
};

enum fbst_array_kind { FBST_ULA = 0, FBST_URA = 1 };

/* How stage 2 (beta_b = A_b^{-1} w_b followed by bhat_b = F_u beta_b) is applied. */
enum fbst_stage2_kind {
  FBST_STAGE2_AUTO = 0,        /* the plan picks GS_IR1 */
  FBST_STAGE2_GS = 1,          /* Gohberg-Semencul with circulant FFTs, then chirp-z (Sec. V); in FP32
                                  its error grows like eps32 * cond(A_b) (~2/delta_rel at broadside) */
  FBST_STAGE2_GS_IR1 = 2,      /* GS plus one FP32 refinement step beta += GS(w - A_b beta) */
  FBST_STAGE2_DENSE_FP32 = 3,  /* precomputed G_b = F_u A_b^{-1} (Sec. III-B), FP32 CUDA cores */
  FBST_STAGE2_DENSE_BF16X3 = 4,/* G_b on tensor cores, split-BF16 (hi*hi + hi*lo + lo*hi), FP32 acc */
  FBST_STAGE2_DENSE_TF32 = 5,  /* G_b on tensor cores in TF32, FP32 accumulate */
  FBST_STAGE2_DENSE_TF32X3 = 6,/* G_b on tensor cores, split TF32 (hi*hi + hi*lo + lo*hi): FP32-class */
  FBST_STAGE2_DENSE_F16X3 = 7  /* G_b on tensor cores, split FP16 (hi*hi + hi*lo + lo*hi) with exact
                                  power-of-two scales per beam of G and per block of w: FP32-class,
                                  at twice the TF32 MMA rate */
};

/* How the plan solves for the stage-2 generators x_b = A_b^{-1} e_0 (Sec. V), in FP64. Both give
 * the same x up to rounding (both are tested against a dense solve). */
enum fbst_generator_solver {
  FBST_GEN_LEVINSON = 0,  /* Levinson recursion, O(L^2) per beam, one CTA per beam */
  FBST_GEN_SUPERFAST = 1  /* doubling Schur algorithm with FFT polynomial products, O(L log^2 L)
                             per beam (the fast generator computation Sec. V points to); L <= 2049 */
};

/* Array and beam grid. M = mx*my elements, B = bx*by beams. A linear array has my = by = 1. */
typedef struct {
  int kind;   /* FBST_ULA or FBST_URA */
  int mx, my; /* elements along x and y */
  int bx, by; /* beams along u and v */
} fbst_geometry;

/* Band and basis parameters (Sec. III-A, Sec. VI). */
typedef struct {
  double frac_bw;     /* fractional bandwidth fb = 2*Omega/f_c, 0 < fb < 2; rounded by the plan
                         to the nearest fraction with denominator <= 1000 (see fbst_info) */
  double epsilon;     /* frequency stretch epsilon >= 1 of Eq. (3); rounded like frac_bw */
  int gamma_num;      /* L = N*gamma_num/gamma_den must be an even integer (Eq. (3), gamma = L/N) */
  int gamma_den;
  double delta;       /* regulariser of Eq. (5): absolute, or relative (see delta_relative) */
  int delta_relative; /* nonzero: the plan uses delta*M*N (M*N is the diagonal of F_b^H F_b) */
  int stage2;         /* enum fbst_stage2_kind */
  int max_blocks;     /* blocks the plan's workspace holds; larger nblk run in chunks (>= 1) */
  int generator_solver; /* enum fbst_generator_solver (0: Levinson) */
} fbst_band;

/* Everything the plan derived from its arguments. */
typedef struct {
  int M, N, B, L;
  int P_time;       /* FFT size of the temporal chirp-z (stage 1a) */
  int S_time;       /* output splits of the temporal chirp-z (1 or 2) */
  int P_space_x;    /* FFT size of the spatial chirp-z along x (the only axis of a linear array) */
  int P_space_y;    /* FFT size of the spatial chirp-z along y (rectangular arrays) */
  int P_gs;         /* circulant size of the Gohberg-Semencul products (>= 2L-1) */
  int P_rec;        /* FFT size of the reconstruction chirp-z F_u */
  int S_rec;        /* input splits of the reconstruction chirp-z (1 or 2) */
  int stage2;       /* resolved enum fbst_stage2_kind */
  double delta;     /* absolute delta used in A_b */
  int64_t eps_num, eps_den; /* epsilon = eps_num/eps_den as used by the plan */
  int64_t fb_num, fb_den;   /* frac_bw = fb_num/fb_den as used by the plan */
  double rho;       /* Omega/(f_c + Omega) = fb/(2+fb): delay per element per unit direction cosine */
  double snapshot_bound; /* right-hand side of Eq. (8) in samples */
  double gamma_bound;    /* right-hand side of Eq. (4) */
  int warn_snapshots;    /* 1 if N does not exceed the Eq. (8) bound */
  int warn_gamma;        /* 1 if gamma does not exceed the Eq. (4) bound */
  size_t table_bytes;     /* device bytes of the plan's tables, held for its lifetime (the plan-time
                             temporaries come and go during fbst_plan) */
  size_t workspace_bytes; /* device bytes of the plan's per-call workspace */
} fbst_info;

/* Host-only: derive the plan parameters of Sec. III-A and Sec. VI (the basis size L = gamma*N and
 * frequency grid of Eq. (3), delta of Eq. (5), the bounds of Eq. (4) and Eq. (8)) and the transform
 * sizes of Sec. IV and Sec. V, without touching a GPU. Same validation as fbst_plan.
 * M and B must equal mx*my and bx*by. Returns FBST_ERR_INVALID / FBST_ERR_UNSUPPORTED on bad
 * input and fills *out otherwise. */
int fbst_derive(const fbst_geometry* g, int M, int N, int B, const fbst_band* band, fbst_info* out);

/* Device-memory allocator of a plan; no counterpart in the paper. alloc returns `bytes` of device
 * memory of the plan's device, 16-byte aligned (256 recommended), usable in stream order on
 * `stream`, or NULL when it has none; free takes back a block that alloc returned, with the same
 * byte count, in stream order on `stream`. ctx is the caller's pointer, passed through. The
 * library calls them only from inside its own entry points, on the calling host thread. */
typedef void* (*fbst_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*fbst_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

/* Build a plan on the current CUDA device: chirp tables and Bluestein kernel spectra (exact
 * integer reduction of the quadratic phases, FP64), Toeplitz generators of every A_b (Sec. V),
 * FP64 Levinson solves for the first column of A_b^{-1}, and either the Gohberg-Semencul spectra
 * or the dense operators G_b = F_u A_b^{-1}. Plan-time kernels run on `stream` and the call
 * synchronises it before returning.
 * Memory: every device block the plan ever holds (its tables and workspace, plan-time
 * temporaries, the staging buffers of fbst_execute_host, fbst_autotune's test input, and the
 * memory of nulling objects built on it) comes from alloc(bytes, stream, ctx) and goes back
 * through free(ptr, bytes, stream, ctx), both ordered on this `stream`, which must stay valid until
 * fbst_destroy. alloc = free = NULL selects cudaMallocAsync / cudaFreeAsync on `stream`; giving
 * only one of them is FBST_ERR_INVALID. When alloc returns NULL the call fails with FBST_ERR_OOM
 * and everything it had obtained is freed again (nothing leaks). */
int fbst_plan(fbst_plan_t* out, const fbst_geometry* g, int M, int N, int B, const fbst_band* band,
              void* stream, fbst_alloc_fn alloc, fbst_free_fn free, void* ctx);

/* fbst_plan for an array whose elements sit at arbitrary positions (Sec. IX, Eq. (16)):
 * positions (host, [M][2] doubles, (x, y) in half wavelengths at f_c + Omega, element m's delay
 * rho*(u*x_m + v*y_m); y = 0 for a linear array; NULL gives the grid, i.e. fbst_plan; element m is
 * the m-th element of y's [M] axis). Off the grid only the element sum of stage 1b changes: it
 * becomes a type-1 non-uniform FFT per frequency: for a linear array each element is spread onto
 * an oversampled grid of nf = pow2(>= 2B) points with a 9-point "exponential of semicircle"
 * kernel, then an nf-point FFT and division by the kernel's Fourier transform; for a rectangular
 * array onto an nf_x x nf_y grid (pow2 >= 2 bx, 2 by) with the 9 x 9 product kernel, then a 2-D
 * FFT and the two axes' factors (kernel error about 1e-8 per axis, below the FP32 rounding). The
 * Toeplitz generators of A_b are direct FP64 sums over the positions. Stage 1a, the generator
 * solves and every stage-2 variant are those of fbst_plan. info.P_space_x (and P_space_y) report
 * the grid sizes. A rectangular array whose grid exceeds 128 x 128 points, or whose kernel would
 * need more than the 227 KB of shared memory (the grid, its FFT buffers and a [B][5] output tile),
 * is FBST_ERR_UNSUPPORTED, and so are nulling and off-grid objects on any such plan; batches
 * accept a linear one. A position that is not finite, or a nonzero y on a linear array, is
 * FBST_ERR_INVALID. */
int fbst_plan_positions(fbst_plan_t* out, const fbst_geometry* g, const double* positions, int M, int N, int B,
                        const fbst_band* band, void* stream, fbst_alloc_fn alloc, fbst_free_fn free, void* ctx);

/* Whole transform: y (device, [nblk][M][N]) -> bhat (device, [nblk][B][N]). nblk = 0 is a no-op.
 * Blocks are independent contiguous batches of N snapshots (Sec. III-A, streaming paragraph). */
int fbst_execute(fbst_plan_t p, const void* y, void* bhat, int nblk, void* stream);

/* The transform of Sec. III-A (as fbst_execute) with HOST buffers (pinned or pageable); the host
 * copies have no counterpart in the paper. Synchronises `stream` before
 * returning, and results are bitwise those of fbst_execute. y is copied in through plan-owned
 * staging memory (allocated on the first call) in block parts that overlap stage 1. If bhat_host
 * is pinned (page-locked, mapped) host memory, stage 2 stores into it directly through its device
 * address; otherwise it is copied out in parts that overlap the rest of stage 2. Two plan-owned
 * copy streams order themselves after `stream`'s earlier work. Errors as fbst_execute, plus
 * FBST_ERR_OOM when the staging allocation fails and FBST_ERR_CUDA when a copy fails
 * (fbst_last_error says why). */
int fbst_execute_host(fbst_plan_t p, const void* y_host, void* bhat_host, int nblk, void* stream);

/* Same result as fbst_execute, for callers that cannot allocate device memory while they run the
 * transform: a real-time receive loop that must never block inside the allocator (cudaMalloc may
 * synchronise the whole device), or a process whose device-memory budget is fixed and checked at
 * start-up. The paper has no counterpart; this is a library convenience. The intermediates live
 * in one 64 MiB static device array of the library instead of the plan's workspace, and the call
 * allocates nothing. The caller still passes y and bhat, and the plan must belong to the current
 * device (FBST_ERR_INVALID otherwise). Rejects (FBST_ERR_INVALID, nothing launched) a call whose
 * intermediates, 8*nblk*(L*M + B*L) bytes, exceed 64 MiB. Its first call on a device looks up the
 * array's address (cudaGetSymbolAddress), so make that first call before any stream capture. All
 * calls share the array and it keeps the last call's contents, so calls that overlap on the GPU
 * race and must be serialised. Not available for the tensor-core stage-2 variants
 * (FBST_ERR_UNSUPPORTED). */
int fbst_execute_noalloc(fbst_plan_t p, const void* y, void* bhat, int nblk, void* stream);

/* The transform of a continuous record in contiguous, overlapping blocks (Sec. III-A: batches of
 * snapshots acquired in sequence may overlap). record (device, [M][T] complex64, sample fastest,
 * 16-byte aligned): block k is samples [k*hop, k*hop + N) of every sensor, read in place;
 * (nblk - 1)*hop + N <= T. out (device, [B][nblk*hop]): each block contributes its central hop
 * output samples [c, c + hop), c = (N - hop)/2, so out[b][k*hop + i] is beam b at record time
 * c + k*hop + i; 1 <= hop <= N with N - hop even. hop = N gives non-overlapping blocks; a smaller
 * hop drops the block edges, where the block's Fourier extension fits worst. The blocks' full
 * outputs pass through plan memory ([max_blocks][B][N], through the plan's allocator on first
 * use). Asynchronous on `stream`; FBST_ERR_INVALID for sizes outside these rules. */
int fbst_execute_stream(fbst_plan_t p, const void* record, long long T, int hop, void* out, int nblk, void* stream);

/* Stage 1 alone, the fan chirp-z of Sec. IV (App. B for rectangular arrays):
 * y (device, [nblk][M][N]) -> w (device, [nblk][B][L]), w_b = F_b^H y. */
int fbst_czt(fbst_plan_t p, const void* y, void* w, int nblk, void* stream);

/* The temporal chirp-z of Sec. IV alone: yhat[blk][ell][m] = sum_n y[blk][m][n] e^{-j omega_ell n}
 * (device, [nblk][L][M], element fastest). Exposed for stage-level testing. */
int fbst_czt_time(fbst_plan_t p, const void* y, void* yhat, int nblk, void* stream);

/* The spatial chirp-z of Sec. IV (App. B) alone: yhat (device, [nblk][L][M], as written by
 * fbst_czt_time) -> w (device, [nblk][B][L]). fbst_czt_time followed by fbst_czt_space equals
 * fbst_czt. Exposed for stage-level testing and timing. */
int fbst_czt_space(fbst_plan_t p, const void* yhat, void* w, int nblk, void* stream);

/* Stage 2 alone (Sec. V): w (device, [nblk][B][L]) -> bhat (device, [nblk][B][N]),
 * bhat_b = F_u (F_b^H F_b + delta I)^{-1} w_b, with the plan's stage-2 variant. */
int fbst_toeplitz_apply(fbst_plan_t p, const void* w, void* bhat, int nblk, void* stream);

/* Failure detection; no counterpart in the paper. Set the limit, in nanoseconds, of each pipeline
 * wait of the plan's tensor-core stage-2 kernels (and of the nulling contraction built on the
 * plan) for later launches; 0 restores the default of 1 s. A wait that runs out makes the kernel
 * record FBST_ERR_TIMEOUT in the plan's status word (read by fbst_sync_status), wait up to 2 s for
 * its own copies and MMAs in flight, free its tensor memory and return; that launch's output is
 * then not valid. A very small limit makes the next launch time out, which tests this path. */
int fbst_set_wait_limit(fbst_plan_t p, uint64_t ns);

/* Calibration; no counterpart in the paper. Measure the FP32 FMA throughput of the current device:
 * one warm-up and one timed launch of a kernel in which every thread of every resident CTA runs
 * independent FMA chains (2 flops each), `iters` x 128 FMAs per thread. sink: device, >= 4 bytes,
 * written only in a case that cannot occur. *tflops receives the measured TFLOP/s and *ms (may be
 * NULL) the timed launch's duration (CUDA events on `stream`, which the call synchronises). */
int fbst_fp32_fma_peak(void* sink, int iters, double* tflops, double* ms, void* stream);

/* Tracing; no counterpart in the paper. From now on record CUDA events (timing enabled) on the
 * call's stream around the three stages of every fbst_execute call: before stage 1a, between 1a
 * and 1b, between 1b and stage 2, after stage 2 (of the call's first chunk when nblk exceeds
 * max_blocks), for the last `capacity` calls (a ring). capacity 0 stops tracing and frees the
 * events; a new capacity drops what was recorded. The events cost four cudaEventRecord calls per
 * traced call and no kernel. Host-side state: calls on one plan from several host threads at once
 * are not supported while tracing. FBST_ERR_INVALID (NULL plan, capacity < 0 or > 2^20),
 * FBST_ERR_OOM, FBST_ERR_CUDA (event creation). */
int fbst_trace_stages(fbst_plan_t p, int capacity);

/* Wait for the traced calls not read yet and write the device time, in milliseconds, of their
 * stage 1a, stage 1b and stage 2 to ms[3*i], ms[3*i + 1], ms[3*i + 2], oldest call first, for at
 * most max_calls calls (ms holds 3*max_calls floats, host memory). Returns the number of calls
 * written (>= 0; the others are dropped) or a negative status: FBST_ERR_INVALID (NULL plan, or ms
 * NULL with max_calls > 0), FBST_ERR_CUDA. */
int fbst_trace_read(fbst_plan_t p, float* ms, int max_calls);

/* Error reporting; no counterpart in the paper. Synchronise `stream`, then return and clear the
 * plan's device status word: FBST_OK, or the
 * error a kernel recorded since the last check (FBST_ERR_TIMEOUT when a bounded device-side wait
 * of the tensor-core kernel gave up; its outputs are then not valid). */
int fbst_sync_status(fbst_plan_t p, void* stream);

/* Copy the derived parameters of a plan (those fbst_derive returns: Sec. III-A, Sec. IV-VI) to the
 * caller's *out. FBST_ERR_INVALID if p or out is NULL. */
int fbst_plan_info(fbst_plan_t p, fbst_info* out);

/* Copy the first column x_b of A_b^{-1} for every beam (the FP64 result of the plan's generator
 * solver, Sec. V) to host memory `x_host` as [B][L] complex128 (interleaved doubles). Exposed for
 * testing. */
int fbst_plan_generators(fbst_plan_t p, void* x_host);

/* Solve again for the generators of Sec. V, x_b = A_b^{-1} e_0 for every beam b of the plan, with
 * the given enum fbst_generator_solver, from the plan's Toeplitz generators a_b (recomputed in
 * FP64, as at plan time). x: device memory, [B][L] complex128 (interleaved doubles), written by
 * the call; the plan's own generators are not changed. Enqueued on `stream` (NULL: the legacy
 * default stream) with a stream-ordered temporary of the plan's allocator (the superfast solver's
 * workspace: one slot of about 18 L complex128 per resident CTA). Errors: FBST_ERR_INVALID (NULL
 * plan or x, unknown method), FBST_ERR_UNSUPPORTED (superfast with L > 2049), FBST_ERR_OOM; a
 * pivot that is not positive records FBST_ERR_NUMERIC for fbst_sync_status. For testing and for
 * timing the two solvers. */
int fbst_solve_generators(fbst_plan_t p, int method, void* x, void* stream);

/* Resource management; no counterpart in the paper. Free the plan and all of its device memory
 * (including that of nulling objects still built on it) through its free function, in stream order
 * on the stream given to fbst_plan. Does not synchronise the device: work that uses the plan on
 * other streams must have finished, or be ordered before the plan's stream, before this call.
 * NULL is OK. */
int fbst_destroy(fbst_plan_t p);

/* Error reporting; no counterpart in the paper. Static human-readable name of a status code (the
 * library owns the string; an unknown code gives "unknown fbst status"). */
const char* fbst_status_string(int status);

/* Error reporting; no counterpart in the paper. Description of the last CUDA failure seen by
 * this host thread ("" if none). The string is owned
 * by the library and stays valid until the next failing call on the same thread. */
const char* fbst_last_error(void);

/* Launch accounting; no counterpart in the paper. Number of kernels one fbst_execute of nblk
 * blocks launches (stage 1 of Sec. IV plus stage 2 of Sec. V); 0 for a NULL plan or nblk <= 0. */
int fbst_launch_count(fbst_plan_t p, int nblk);

/* ---------------------------------------------------------------------------------------------
 * Batches of independent arrays. Blocks, requests and whole arrays are independent (Sec. III-A
 * streaming remark; Sec. VI on parallel execution over beams and frequency pairs), so many plans of
 * different sizes can run together. A batch run groups the plans' work by kernel and transform
 * size into a few launches that spread all their work items over the whole GPU, and replays that
 * launch sequence as a CUDA graph.
 * ------------------------------------------------------------------------------------------- */
typedef struct fbst_batch_s* fbst_batch_t;

/* Group `count` distinct plans into a batch (the batch keeps pointers; the plans must outlive
 * it and must not run elsewhere while a batch run using them is in flight). The grouping has no
 * counterpart in the paper; each plan still computes the transform of Sec. III-A. FBST_ERR_INVALID
 * for count < 1, a NULL or repeated plan. */
int fbst_batch_create(fbst_batch_t* out, const fbst_plan_t* plans, int count);

/* Run plan i on nblk[i] blocks (0 <= nblk[i] <= that plan's max_blocks): y[i] ([nblk][M][N]) ->
 * bhat[i] ([nblk][B][N]), device pointers, asynchronous on `stream`. The first run with a given
 * set of pointers and block counts launches eagerly and captures the launch sequence into a CUDA
 * graph; later runs with the same arguments replay the graph. Results equal per-plan fbst_execute. */
int fbst_batch_execute(fbst_batch_t b, const void* const* y, void* const* bhat, const int* nblk, void* stream);

/* Same grouped launches as fbst_batch_execute, enqueued directly without capturing a graph (for
 * callers whose pointer sets change on every call, such as a continuous-batching server). */
int fbst_batch_enqueue(fbst_batch_t b, const void* const* y, void* const* bhat, const int* nblk, void* stream);

/* Launch accounting; no counterpart in the paper. Kernels in one graph replay of the batch (0
 * before the first run). */
int fbst_batch_launch_count(fbst_batch_t b);

/* Resource management; no counterpart in the paper. Release the batch and its captured graph
 * (not its plans). NULL is OK. */
int fbst_batch_destroy(fbst_batch_t b);

/* ---------------------------------------------------------------------------------------------
 * Launch shapes of the two stage-1 kernels: the Stockham radix (elements per thread, E) and the
 * transforms per CTA (G). Not part of the method; performance only, results stay within rounding.
 * ------------------------------------------------------------------------------------------- */
/* Time every compiled shape of the temporal and the spatial chirp-z kernels of Sec. IV for this
 * plan on
 * nblk blocks (on the plan's workspace and a temporary input buffer it allocates), keep the
 * fastest in the plan, and write {time_E, time_G, space_E, space_G} to shapes4 (may be NULL).
 * Synchronises `stream`. Not allowed during stream capture. */
int fbst_autotune(fbst_plan_t p, int nblk, void* stream, int* shapes4);

/* Set the shapes of the Sec. IV kernels explicitly ({0, 0} restores the built-in default for
 * that kernel);
 * FBST_ERR_UNSUPPORTED if no kernel of that shape is compiled for the plan's transform size. */
int fbst_set_shapes(fbst_plan_t p, int time_E, int time_G, int space_E, int space_G);

/* Read the shapes of the Sec. IV kernels in use into shapes4: {time_E, time_G, space_E, space_G}. */
int fbst_get_shapes(fbst_plan_t p, int* shapes4);

/* ---------------------------------------------------------------------------------------------
 * Off-grid beams (Sec. VIII-A). A direction (u, v) between the grid beams of a plan gets its beam
 * vector by interpolating the stage-1 vectors w_b of the grid beams around it: a natural cubic
 * spline in the direction cosine through the K grid beams nearest to u (K/2 on each side of the
 * interval that holds u, moved inward at the ends of the grid; the paper uses 8), and for a
 * rectangular array the tensor product of the splines along u and v (K x K grid beams). Then the
 * off-grid direction's own regularised least-squares beam (Eq. (5)-(7)):
 *     bhat*_k = F_u (F*_k^H F*_k + delta I)^{-1} w*_k,   w*_k = sum_i c_{k,i} w_{b_i},
 * applied by Gohberg-Semencul with one FP32 refinement step (Sec. V) from FP64 plan-time spectra
 * (generators of every A*_k from their closed form, FP64 Levinson). The interpolation weights are
 * computed on the host in FP64 and rounded once. w*_k approximates the exact F*_k^H y; the distance
 * between the two is a property of the spline, not an error of this library.
 * ------------------------------------------------------------------------------------------- */
typedef struct fbst_offgrid_s* fbst_offgrid_t;

/* Build the off-grid beams of `ndir` directions (host array `directions`, [ndir][2] direction
 * cosines (u, v), |u|, |v| <= 1; v must be 0 for a linear array) for plan `p`, which must belong to
 * the current device; K (2..16) grid beams per axis enter each interpolation (fewer if the grid
 * has fewer). Plan-time kernels run on `stream`, which the call synchronises. Device memory, all
 * through the plan's allocator: 24*ndir*P_gs + 8*max_blocks*ndir*L bytes and small tables. The plan
 * must outlive the object and the two must not run concurrently (they share the plan's workspace).
 * FBST_ERR_INVALID for bad arguments, FBST_ERR_OOM / FBST_ERR_CUDA on allocation or launch failure,
 * FBST_ERR_NUMERIC if a direction's A is not numerically positive definite. */
int fbst_offgrid_create(fbst_offgrid_t* out, fbst_plan_t p, const double* directions, int ndir, int K,
                        void* stream);

/* The interpolation alone: w (device, [nblk][B][L], as written by fbst_czt) -> wstar (device,
 * [nblk][ndir][L]). Asynchronous on `stream`; pointers 16-byte aligned (else FBST_ERR_INVALID). */
int fbst_offgrid_interpolate(fbst_offgrid_t o, const void* w, void* wstar, int nblk, void* stream);

/* Off-grid beams from the stage-1 output: w (device, [nblk][B][L]) -> bstar (device,
 * [nblk][ndir][N]), interpolation then the directions' stage 2. Asynchronous on `stream`. */
int fbst_offgrid_apply(fbst_offgrid_t o, const void* w, void* bstar, int nblk, void* stream);

/* The whole off-grid transform: y (device, [nblk][M][N]) -> bstar (device, [nblk][ndir][N]) with
 * the plan's stage 1, the interpolation and the directions' stage 2. Asynchronous on `stream`;
 * errors as fbst_execute. */
int fbst_offgrid_execute(fbst_offgrid_t o, const void* y, void* bstar, int nblk, void* stream);

/* Resource management; no counterpart in the paper. Free the object's device memory through the
 * plan's free function (stream-ordered on the plan's stream; work that uses the object must have
 * finished). NULL is OK. */
int fbst_offgrid_destroy(fbst_offgrid_t o);

/* ---------------------------------------------------------------------------------------------
 * Beamspace interference nulling (Sec. VIII-B, Eq. (14)). For interferer beams p_1..p_P of a plan's
 * grid, every output beam b of that plan becomes
 *     bhat_b = F_u A_b^{-1} ( w_b - sum_j F_b^H F_{p_j} A_{p_j}^{-1} w_{p_j} ),   w = F^H y,
 * the paper's G_{b,p} w_p with G_{b,p} = F_b^H F_p (F_p^H F_p + delta I)^{-1}. By the derivation of
 * Eq. (14) this is the plain transform of the measurements after each interferer's regularised
 * projection y - F_p (F_p^H F_p + delta I)^{-1} F_p^H y has been subtracted. The nulling object
 * holds, in device memory, every G_{b,p_j} (B x L x P*L complex64), built once in FP64: each row of
 * F_b^H F_{p_j} from its closed form (exact integer phase reduction), times A_{p_j}^{-1} by the
 * FP64 Gohberg-Semencul apply with the plan's FP64 generators, rounded once. (Applying the two
 * factors at run time would pass A_{p_j}^{-1} w_{p_j} through FP32, and A_p's condition number,
 * about 2/delta_rel, would reach the nulled beams.) At run time the contraction of G with the
 * interferers' stage-1 vectors runs on the split-TF32 tensor-core kernel of the dense stage 2 or on
 * its FP32 CUDA-core kernel.
 * ------------------------------------------------------------------------------------------- */
typedef struct fbst_null_s* fbst_null_t;

typedef enum {
  FBST_NULL_TF32X3 = 0,  /* contraction on the tensor cores, split TF32 (FP32-class accuracy) */
  FBST_NULL_FP32 = 1     /* contraction on the FP32 CUDA cores */
} fbst_null_contraction;

/* Build the nulling of `P` interferer beams (1 <= P <= 16; distinct grid indices in [0, B), read
 * from the host array `interferers`) for plan `p`, on the current device; plan-time kernels run
 * on `stream`, which the call synchronises. The plan must outlive the nulling object, and the two
 * must not run concurrently (they share the plan's workspace and status word). Device memory,
 * all obtained through the plan's allocator (see fbst_plan): 8*B*L*P*L bytes of operator (held
 * once; twice during the call), 32*P*P_gs bytes of spectra, 8*max_blocks*(P*L + B*L) bytes of
 * workspace. Building G costs B*L*P FP64
 * Gohberg-Semencul applies (6 FFTs of P_gs each).
 * FBST_ERR_INVALID for bad arguments, FBST_ERR_UNSUPPORTED when P*L is not a multiple of 8 for the
 * tensor-core contraction or the exact phase reductions would leave 64-bit range, FBST_ERR_OOM /
 * FBST_ERR_CUDA on allocation or launch failure, FBST_ERR_NUMERIC if a generator is not usable. */
int fbst_null_create(fbst_null_t* out, fbst_plan_t p, const int* interferers, int P, int contraction,
                     void* stream);

/* fbst_null_create for interferers at arbitrary directions (Sec. VIII-B: exact alignment of the
 * interference directions with the grid is not required). directions: host [P][2] direction
 * cosines (u, v), |u|, |v| <= 1, v = 0 for a linear array. Each interferer's vector w_p is
 * interpolated from the grid beams' stage-1 vectors as in fbst_offgrid_create (a natural cubic
 * spline through the K grid beams per axis around the direction, 2 <= K <= 16; Sec. VIII-A), and
 * G_{b,p} = F_b^H F_p A_p^{-1} uses the direction's own F_p: the cross Gram rows from their closed
 * form in FP64 and A_p^{-1} from the direction's FP64 Levinson generator. The plan must belong to
 * the current device. Otherwise as fbst_null_create. */
int fbst_null_create_directions(fbst_null_t* out, fbst_plan_t p, const double* directions, int P, int K,
                                int contraction, void* stream);

/* The time-domain form of the nulling (Sec. VIII-B, Eq. (15)) for P grid interferer beams: each
 * interferer's beam y_p = F_x A_p^{-1} w_p over a broader reconstruction interval, the 2L samples
 * t = -(2L - N)/2 .. (2L + N)/2 - 1 centred on the block (F_x = F_u of Eq. (7) on that interval, of
 * full column rank and well conditioned; an interval of only L samples is square but numerically
 * singular for L in the hundreds), is mapped by G'_{b,p} = F_u H_{b,p} F_x^+,
 * H_{b,p} = A_b^{-1} F_b^H F_p, and subtracted from the plain beam y_b over the block's N samples.
 * The object holds, built in FP64: the cross Gram matrices F_b^H F_p ([B][L][P*L], complex64),
 * F_x A_p^{-1} ([P][2L][L], kept in FP64; the interferers' beams are summed from it in FP64, since
 * its entries are of the size of ||A_p^{-1}|| and cancel down to the beam) and
 * F_x^+ = (F_x^H F_x)^{-1} F_x^H ([P][L][2L], complex64); G'_{b,p} is applied factor by factor (F_x^+,
 * the cross Gram contraction, the plan's stage 2). With F_x of full column rank the result equals
 * Eq. (14) up to rounding. Requires N even and L <= 1024 (FBST_ERR_UNSUPPORTED otherwise); device
 * memory 8*B*L*P*L + 48*P*L*L bytes plus 8*max_blocks*(3*P*L + B*L + B*N) of workspace. Otherwise
 * as fbst_null_create; fbst_null_apply is FBST_ERR_UNSUPPORTED on such an object, fbst_null_execute
 * runs the time-domain form. */
int fbst_null_create_time(fbst_null_t* out, fbst_plan_t p, const int* interferers, int P, int contraction,
                          void* stream);

/* Eq. (15) on time-domain beams (an object of fbst_null_create_time): y (device, [nblk][B][N], the
 * plain beams over each block) and y_int (device, [nblk][P][2L], the interferers' beams over the
 * broader interval, in the order of the object's interferers) -> out (device, [nblk][B][N]),
 * out_b = y_b - sum_p G'_{b,p} y_p. out may equal y. Asynchronous on `stream`; pointers 16-byte
 * aligned (else FBST_ERR_INVALID). FBST_ERR_UNSUPPORTED on an object of the other forms. */
int fbst_null_apply_time(fbst_null_t n, const void* y, const void* y_int, void* out, int nblk, void* stream);

/* The bracket of Eq. (14) alone: w (device, [nblk][B][L], as fbst_czt writes it) ->
 * wt (device, [nblk][B][L]), wt_b = w_b - sum_j F_b^H F_{p_j} A_{p_j}^{-1} w_{p_j}. wt may equal w
 * (in place); otherwise the two must not overlap. Asynchronous on `stream`; both pointers 16-byte
 * aligned (else FBST_ERR_INVALID, nothing launched). */
int fbst_null_apply(fbst_null_t n, const void* w, void* wt, int nblk, void* stream);

/* The whole nulled transform: y (device, [nblk][M][N]) -> bhat (device, [nblk][B][N]) with the
 * plan's stage 1, the bracket of Eq. (14) and the plan's stage 2. Asynchronous on `stream`;
 * errors as fbst_execute; device-side errors are read with fbst_sync_status on the plan. */
int fbst_null_execute(fbst_null_t n, const void* y, void* bhat, int nblk, void* stream);

/* Launch accounting; no counterpart in the paper. Kernels one fbst_null_execute of nblk blocks
 * launches (fbst_null_apply launches 3 per chunk of max_blocks); 0 for NULL or nblk <= 0. */
int fbst_null_launch_count(fbst_null_t n, int nblk);

/* Resource management; no counterpart in the paper. Free the nulling object's device memory
 * (not the plan) through the plan's free function, in stream order on the plan's stream. Does not
 * synchronise the device: work that uses the object must have finished, or be ordered before the
 * plan's stream, before this call. NULL is OK. */
int fbst_null_destroy(fbst_null_t n);

#ifdef __cplusplus
}
#endif

#endif /* FBST_H */
