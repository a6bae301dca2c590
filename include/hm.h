/*
 * hm.h -- C ABI of libhm: compressed hierarchical-matrix products on one GB300.
 *
 * Operation (eqn. mvm, Sec. 3, extended by beta):
 *     y := alpha * M * x + beta * y      (and alpha * M^H * x + beta * y)
 * for an H-, uniform-H (UH) or H^2-matrix M (Sec. 2.2-2.4) whose dense
 * leaves, low-rank factors, cluster bases, coupling and transfer matrices are
 * stored in the floating point compressed formats of Sec. 4 (AFLP or FPX,
 * direct compression at eps, VALR per column from the singular values) and are
 * decompressed inside the GPU kernels during the product.
 *
 * Conventions shared by every entry point:
 *  - Every call returns an hm_status; nothing is thrown across the ABI.
 *  - "host" pointers are ordinary CPU memory, "device" pointers are CUDA
 *    global memory of the current device.  The caller owns every pointer it
 *    passes; the library owns the hm_matrix and everything reachable from it.
 *  - Vectors are FP64 in the ORIGINAL point order, column-major with a leading
 *    dimension (ld >= n) and nrhs columns.
 *  - GPU work is enqueued on the caller's stream (a cudaStream_t passed as
 *    void*, NULL = legacy default stream) and never synchronised by the
 *    library unless the entry point says so.
 */
#ifndef HM_H
#define HM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hm_matrix hm_matrix;            /* opaque, library-owned */

typedef enum {
  HM_OK = 0,
  HM_ERR_ARG = 1,        /* invalid argument (null pointer, size, enum value) */
  HM_ERR_OOM = 2,        /* host or device allocation failed */
  HM_ERR_CUDA = 3,       /* a CUDA runtime call failed */
  HM_ERR_STATE = 4,      /* call order violated (e.g. matvec before compress) */
  HM_ERR_TIMEOUT = 5,    /* a device-side wait ran out of iterations */
  HM_ERR_IO = 6,         /* file could not be read or written */
  HM_ERR_DEVICE = 7,     /* a kernel latched a bounds / format error */
  HM_ERR_UNSUPPORTED = 8, /* data outside what the kernels decode (see hm_compress) */
  HM_ERR_CAPACITY = 9     /* request larger than a fixed limit (hm_matvec_host_noalloc's scratch,
                             hm_compress's addressing) */
} hm_status;

/* UH_SEP: uniform-H with separate row and column coupling matrices per block,
 * S = Sr Sc^H (the variant discussed after Alg. 5): the product takes
 * u_b = Sc_b^H s_sigma per block, then t_tau = sum_b Sr_b u_b. */
typedef enum { HM_FMT_H = 0, HM_FMT_UH = 1, HM_FMT_H2 = 2, HM_FMT_UH_SEP = 3 } hm_format;
/* Admissibility of the block tree (Def. Block Tree and the remark after Def.
 * H-Matrix): STANDARD min(diam t, diam s) <= eta dist(t, s); HODLR off-diagonal
 * (every block of two distinct clusters is low rank, dense blocks only on the
 * diagonal); BLR a single level (only blocks of leaf clusters are tested with the
 * standard condition, larger blocks are always subdivided). */
typedef enum { HM_ADM_STANDARD = 0, HM_ADM_HODLR = 1, HM_ADM_BLR = 2 } hm_adm;
typedef enum { HM_CODEC_NONE = 0, HM_CODEC_AFLP = 1, HM_CODEC_FPX = 2 } hm_codec;
/* Matrix entries of the model problems (point-kernel stand-ins for the
 * Galerkin single-layer matrix of Sec. 2.1):
 *   LAPLACE   a_ij = 1 / (4 pi |p_i - p_j|), a_ii = 1 / (4 pi h);
 *   MATERN15  a_ij = (1 + sqrt3 r / l) exp(-sqrt3 r / l), r = |p_i - p_j|, a_ii = 1;
 *   LAPLACE_W w_i times the LAPLACE entry, w_i = 1 + x_i / 2 (x_i the first
 *             coordinate of point i): diag(w) A, a non-symmetric matrix for
 *             checks of the adjoint product. */
typedef enum { HM_KERNEL_LAPLACE = 0, HM_KERNEL_MATERN15 = 1, HM_KERNEL_LAPLACE_W = 2 } hm_kernel;

typedef struct {
  int32_t kernel;      /* hm_kernel */
  double kparam;       /* Laplace (and LAPLACE_W): diagonal spacing h (<= 0: sqrt(4 pi / n));
                          Matern: length scale (<= 0: 0.1) */
  int32_t leaf_size;   /* cluster tree leaf size (Def. Cluster Tree), 1..128 */
  double eta;          /* standard admissibility parameter, > 0 */
  int32_t format;      /* hm_format */
  double eps_build;    /* low-rank accuracy eps (eqn. epsilon), 0 < eps < 1 */
  int32_t nthreads;    /* host threads for construction (<= 0: all cores) */
  int32_t adm;         /* hm_adm: admissibility condition (0 = standard) */
} hm_build_params;

/*
 * hm_build -- construct M on the host (Sec. 2): cluster tree by geometric
 * bisection, block tree with the admissibility of prm->adm (standard, HODLR or
 * BLR), dense leaves, low-rank blocks (ACA + SVD recompression, truncated at
 * sigma_k <= eps*sigma_0), and for UH / UH_SEP / H^2 the shared / nested cluster
 * bases and couplings (UH_SEP: the two factors of every coupling).
 *   pts : host, n x 3 FP64, row-major (x0 y0 z0 x1 ...); copied.
 *   out : receives a new matrix (FP64 host copy; nothing on the GPU yet).
 * Errors: HM_ERR_ARG for null pointers, n < 1 or invalid parameters,
 *         HM_ERR_OOM if host memory runs out.
 */
hm_status hm_build(const hm_build_params* prm, const double* pts, int64_t n, hm_matrix** out);

/*
 * hm_compress -- pack M for the GPU (Sec. 4.1, 4.2) and upload it.
 *   eps   : compression accuracy (m_eps = ceil(-log2 eps)), 0 < eps < 1.
 *   codec : HM_CODEC_NONE (FP64, the uncompressed baseline), AFLP or FPX.
 *   valr  : nonzero = per-column accuracy from the singular values (VALR) for
 *           low-rank factors and cluster bases; zero = direct compression at eps.
 * May be called again (other eps / codec): the previous device copy is freed.
 * Synchronises the device.  Errors: HM_ERR_ARG, HM_ERR_OOM, HM_ERR_CUDA,
 * HM_ERR_UNSUPPORTED if a value range exceeds what the kernels decode
 * (AFLP dynamic range >= 2^127, or |v| >= 2^127), HM_ERR_CAPACITY if the
 * packed form exceeds the library's addressing (64 GiB of packed payload:
 * copy descriptors hold offset / 16 in 32 bits; 2^31 vector entries) or its
 * layout (H^2 cluster bases of rank > 128: a sweep chunk holds <= 128
 * coefficients).
 */
hm_status hm_compress(hm_matrix* m, double eps, int32_t codec, int32_t valr);

/*
 * hm_matvec -- y := alpha*M*x + beta*y on the GPU, stream-ordered, no sync.
 *   x : device, FP64, n x nrhs, leading dimension ldx >= n; read only.
 *   y : device, FP64, n x nrhs, leading dimension ldy >= n; must not overlap x.
 *   nrhs : 1..64 right-hand sides.
 *   stream : cudaStream_t as void* (NULL = default stream).
 * Concurrent calls on one matrix must be ordered by the caller (they share the
 * matrix's workspace).  Device-side errors are latched, see hm_sync_status.
 * Errors: HM_ERR_ARG, HM_ERR_STATE (not compressed), HM_ERR_CUDA (launch).
 */
hm_status hm_matvec(hm_matrix* m, double alpha, const double* x, int64_t ldx, double beta,
                    double* y, int64_t ldy, int64_t nrhs, void* stream);

/*
 * hm_matvec_adjoint -- y := alpha*M^H*x + beta*y (the remark after Alg. 3: the
 * adjoint product runs over the block columns; the data are real, so
 * M^H = M^T).  Same arguments, layout, stream semantics and errors as
 * hm_matvec.  The first call builds the transposed matrix on the host (blocks
 * (t, s) -> (s, t): W and X swapped, dense blocks and couplings transposed, row
 * and column bases exchanged), compresses it with the eps / codec / valr of the
 * last hm_compress -- the same codes, rearranged -- and uploads it; this first
 * call synchronises the stream and needs host and device memory about as large
 * as m's own.  Later calls reuse it until the next hm_compress or hm_free.  The
 * transposed matrix follows m's hm_graph and hm_persistent settings and runs
 * launch shape 0 (hm_autotune tunes m only).
 */
hm_status hm_matvec_adjoint(hm_matrix* m, double alpha, const double* x, int64_t ldx, double beta,
                            double* y, int64_t ldy, int64_t nrhs, void* stream);

/*
 * hm_matvec_host -- the same product on HOST buffers: copies x and y to the
 * device, runs hm_matvec, copies y back, and synchronises the stream.
 * x, y : host FP64 (n x nrhs, ld n, column-major).  Uses library-owned
 * device buffers.  Errors as hm_matvec plus HM_ERR_OOM.
 */
hm_status hm_matvec_host(hm_matrix* m, double alpha, const double* x, double beta, double* y,
                         int64_t nrhs, void* stream);

/*
 * hm_graph -- enable (nonzero) or disable CUDA-graph replay of hm_matvec.
 * When enabled, the first hm_matvec with a given (x, y, ldx, ldy, nrhs,
 * alpha, beta) captures its whole kernel sequence on a library-owned stream
 * into a CUDA graph; later calls with the same arguments launch that graph on
 * the caller's stream (one launch instead of one per kernel).  A call with
 * other arguments re-captures.  hm_compress discards the graph.  Profiling
 * (hm_profile) bypasses the graph.  Errors: HM_ERR_ARG.
 */
hm_status hm_graph(hm_matrix* m, int32_t enable);

/*
 * hm_persistent -- how the launches of one product run (the batching form).
 *   0: one kernel launch per step (gather, column dots, segment sums, fan-outs,
 *      row chunks), chained on the stream;
 *   1 (the default): as 0, but every run of two or more consecutive row-chunk
 *      launches (the row-chunk form of Alg. 3 / 5 / 7 and the sweeps of Alg. 6 /
 *      7, one launch per tree level) executes as the phases of ONE cooperative
 *      launch with one block per SM, each piece waiting (bounded) only for the
 *      coefficient chunks it reads;
 *   2: the whole product -- every step of a1-a10, forward, coupling and backward
 *      passes included -- as ONE cooperative launch with one block per SM: the
 *      steps are its phases, separated by grid barriers (bounded waits), the
 *      runs of row-chunk steps as in 1.
 * A wait that runs out latches HM_ERR_TIMEOUT (hm_sync_status).  Modes 1 and 2
 * use the warp ranges of launch shape 0 whatever hm_autotune chose, and their
 * results equal mode 0 with all shapes 0 bit for bit.  Profiling (hm_profile)
 * always runs mode 0.  Errors: HM_ERR_ARG (enable outside 0..2).
 */
hm_status hm_persistent(hm_matrix* m, int32_t enable);
/* hm_persistent_mode -- the mode in use (0, 1 or 2; hm_autotune may change it). */
hm_status hm_persistent_mode(const hm_matrix* m, int32_t* mode);

/*
 * hm_set_multi_rhs_engine -- how the row-chunk steps of multi-RHS panels (the
 * precision / multi-RHS form, FP32 tier) multiply:
 *   0: tensor cores (tcgen05) -- each decoded value and multiplier cut into
 *      three exact BF16 limbs in shared memory, the limb products of order <= 2
 *      accumulated in TMEM (FP32, orders 0 and 1 + 2 apart);
 *   1 (the default): FP32 pipes -- one FP32 FMA per product, as the single-RHS
 *      kernels, for chunks of at most 64 rows (wider chunks as 0).
 * Both sum per piece in FP32 and across pieces in float-float; results differ
 * only in rounding.  The column dots of a panel run on the FP32 pipes either
 * way.  hm_autotune times both engines on an RP-wide panel and keeps the faster.
 * Errors: HM_ERR_ARG (engine outside 0..1).
 */
hm_status hm_set_multi_rhs_engine(hm_matrix* m, int32_t engine);
/* hm_multi_rhs_engine -- the engine in use (0 or 1). */
hm_status hm_multi_rhs_engine(const hm_matrix* m, int32_t* engine);

/*
 * hm_save -- write m to the file `path`: the built matrix (cluster tree, block
 * tree, dense leaves, low-rank factors, cluster bases, couplings and transfer
 * matrices, FP64, as hm_build made them) and, if m is compressed, the eps /
 * codec / valr of its last hm_compress.  The packed device form is not written
 * (its layout depends on the GPU); hm_load rebuilds it.  Host only, no sync.
 * The format is little-endian with a magic and a version number.
 * Errors: HM_ERR_ARG (null), HM_ERR_IO (the file cannot be written).
 */
hm_status hm_save(const hm_matrix* m, const char* path);

/*
 * hm_load -- read a matrix written by hm_save into a new hm_matrix (*out).  If
 * the saved matrix was compressed, hm_compress runs with the saved settings on
 * the current device, so that the loaded matrix gives the saved one's product
 * bit for bit on the same GPU; an uncompressed one needs no GPU.
 * Errors: HM_ERR_ARG (null), HM_ERR_IO (cannot be read, wrong magic or
 * version, truncated, trailing bytes, or indices out of range), HM_ERR_OOM,
 * and the errors of hm_compress.
 */
hm_status hm_load(const char* path, hm_matrix** out);

/* hm_free -- release host and device memory of m (NULL is accepted). */
hm_status hm_free(hm_matrix* m);

typedef struct {
  int64_t n;                /* matrix dimension */
  int32_t format, codec, valr;
  double eps;               /* accuracy of the last hm_compress (0 if none) */
  int64_t nclusters, nleaves, nblocks, nlowrank, ndense;
  int32_t depth, max_rank;
  int64_t bytes_fp64;       /* FP64 bytes of the same data (uncompressed) */
  int64_t bytes_payload;    /* packed value bytes on the device (with padding) */
  int64_t bytes_values;     /* packed value bytes without padding (algorithmic) */
  int64_t bytes_meta;       /* headers, descriptors, work lists on the device */
  int64_t bytes_workspace;  /* per-product workspace on the device */
  int64_t bytes_lowrank_fp64; /* FP64 bytes of low-rank factors / bases */
  int64_t bytes_dense_fp64;   /* FP64 bytes of dense leaves */
  int64_t nlaunches;        /* kernels launched by one hm_matvec with nrhs = 1 */
  int32_t tier;             /* 0: FP32 arithmetic, 1: float-float (eps <= 2^-22 or NONE) */
  int64_t nunits;           /* packed units (column-dot pieces, then row-chunk pieces) */
  int64_t bytes_inline_meta; /* per-unit headers and per-column decode parameters in the payload */
  int64_t bytes_alg;        /* algorithmic bytes of one product per right-hand side: packed codes
                               (bytes_values) + bytes_inline_meta + 24 n (x read, y read and
                               written, FP64) + 16 per coefficient of the coefficient vectors
                               (t_b / s / t, written once and read once) */
  int64_t bytes_by_width[8]; /* packed code bytes by code width B = 1 .. 8 (VALR and direct widths) */
} hm_info_t;

/* hm_info -- sizes and counts of m.  Errors: HM_ERR_ARG. */
hm_status hm_info(const hm_matrix* m, hm_info_t* out);

/* hm_status_str -- static English text of a status code. */
const char* hm_status_str(hm_status s);

/*
 * hm_sync_status -- synchronise `stream`, then read and clear the matrix's
 * device error word.  Returns HM_ERR_DEVICE / HM_ERR_TIMEOUT if a kernel
 * latched an error since the last call, HM_OK otherwise.
 */
hm_status hm_sync_status(hm_matrix* m, void* stream);

/*
 * hm_structure -- export the cluster tree and block tree (host buffers).
 *   perm      : n int64, perm[position] = original index (may be NULL).
 *   clusters  : nclusters x 4 int64 rows (start, end, level, parent) (may be NULL).
 *   blocks    : nblocks x 3 int64 rows (row cluster, col cluster, admissible)
 *               in depth-first block-tree order (may be NULL).
 *   ranks     : nblocks int32, rank of each low-rank block, -1 for dense (may be NULL).
 */
hm_status hm_structure(const hm_matrix* m, int64_t* perm, int64_t* clusters, int64_t* blocks,
                       int32_t* ranks);

/*
 * Codec entry points (Sec. 4.1).  A packed array of n values with one header
 * is n codes of B bytes each, little-endian, value-contiguous.
 *   hdr[0..3] = B, format (0 FPX-e8, 1 FPX-e11, 2 AFLP, 3 raw FP64), e, m (m' for AFLP)
 *   vmin      = AFLP scale (1 for FPX / raw)
 */
typedef struct { int32_t B, fmt, e, m; double vmin; } hm_codec_header;

/*
 * hm_codec_encode -- host: compress n FP64 values (host, contiguous) with
 * `codec` (AFLP or FPX) at accuracy key (AFLP: m requested mantissa bits;
 * FPX: table row of the key).  out: host, capacity cap bytes (>= 8n suffices).
 * The header reports the format actually used: AFLP stores raw FP64 when
 * 1 + m' + e > 56 or when s = |v|/vmin + 1 leaves the FP64 range; an FPX e8
 * row moves to e11 m28 when a value lies outside the FP32 normal range, and an
 * e11 row to the exact e11 m52 when a value rounds past the FP64 maximum.
 * Errors: HM_ERR_ARG (null, n < 0, key outside 0..60, cap too small, NaN/Inf).
 */
hm_status hm_codec_encode(const double* v, int64_t n, int32_t codec, int32_t key, uint8_t* out,
                          int64_t cap, hm_codec_header* hdr);

/*
 * hm_codec_decode -- device (kernel K0): decode n packed values (device bytes,
 * n*B long) into FP64 (device).  Bit-exact: AFLP uses fl(fl(s-1)*vmin).
 * Stream-ordered, no sync.  Errors: HM_ERR_ARG, HM_ERR_CUDA.
 */
hm_status hm_codec_decode(const uint8_t* packed, int64_t n, const hm_codec_header* hdr,
                          double* out, void* stream);

/*
 * Launch shapes and the autotuner (the batching form: one tuned launch per
 * phase).  Each column-dot and row-chunk launch of a product is split into
 * per-warp ranges of about equal bytes for every launch shape (warps per block
 * x shared-memory stages per warp: 0 = 16 x 3, 1 = 12 x 4, 2 = 8 x 6; one
 * block per SM); which shape a launch uses does not change its result beyond
 * the order of summation inside a chunk.
 * hm_autotune -- time every shape of every such launch `reps` times on
 *   `stream` (on internal zero vectors) and keep the fastest per launch; then
 *   time the whole product in each hm_persistent mode and keep the fastest;
 *   in the FP32 tier also time an RP-wide multi-RHS panel with each
 *   hm_set_multi_rhs_engine engine and keep the faster (two more n x RP
 *   buffers for the call).
 *   Allocates two n-vectors for the duration of the call, synchronises the
 *   stream, and discards a captured graph.  Errors: HM_ERR_ARG (reps outside
 *   1..1000), HM_ERR_STATE (not compressed), HM_ERR_CUDA.
 * hm_launch_shapes -- the shape of every launch of one product (-1 for the
 *   gather and segment-sum launches) in shapes[0 .. min(cap, count)); count =
 *   number of launches.  Errors: HM_ERR_ARG.
 * hm_set_launch_shapes -- use `shape` (0..2) for every launch (the default
 *   after hm_compress is 0).  Errors: HM_ERR_ARG.
 */
hm_status hm_autotune(hm_matrix* m, int32_t reps, void* stream);
hm_status hm_launch_shapes(const hm_matrix* m, int32_t* shapes, int32_t cap, int32_t* count);
hm_status hm_set_launch_shapes(hm_matrix* m, int32_t shape);

/*
 * Tuning records: what hm_autotune chose for a compressed matrix (every
 * launch's shape, the hm_persistent mode, the multi-RHS engine), as an opaque
 * int32 array, so that a caller can keep it per device and apply it to an
 * identical matrix later without timing again.  The record carries a
 * fingerprint of the device (SM count, name) and of the matrix's launch
 * program (tier, every launch's kind, output mode, units and warp ranges).
 * hm_tuning -- writes the record to rec[0 .. min(cap, *len)); *len = its length
 *   (5 + launches + 2).  Host only.  Errors: HM_ERR_ARG, HM_ERR_STATE (not
 *   compressed).
 * hm_set_tuning -- applies a record; HM_ERR_ARG if it was taken on another
 *   device or program (fingerprint or launch count differ) or holds a value out
 *   of range; HM_ERR_STATE if m is not compressed.  Discards a captured graph.
 */
hm_status hm_tuning(const hm_matrix* m, int32_t* rec, int32_t cap, int32_t* len);
hm_status hm_set_tuning(hm_matrix* m, const int32_t* rec, int32_t len);

/*
 * Kernel profiling.  hm_profile(m, 1) makes every later hm_matvec record a
 * CUDA event pair around each of its kernel launches, on the caller's stream;
 * hm_profile_read synchronises those events, returns per kernel kind the
 * summed duration, the launch count and the algorithmic bytes those launches
 * move (packed values, format words, descriptors, vector reads and writes),
 * and clears the record.  Kinds: 0 gather, 1 column dots (phase A),
 * 2 segment sums, 3 row chunks (phase C / couplings / sweeps), 4 multiplier
 * fan-out (copies the coefficients each row-chunk piece multiplies into
 * contiguous runs; where the column dots and segment sums right before it wrote
 * every such coefficient -- the H product -- the segment-sum launch fills
 * these slots itself and kind 4 has no launch).  out : host array of nout
 * (<= 5) entries.
 * Errors: HM_ERR_ARG, HM_ERR_CUDA.
 */
typedef struct { double ms; int64_t launches; int64_t bytes; } hm_kernel_stat;
hm_status hm_profile(hm_matrix* m, int32_t enable);
hm_status hm_profile_read(hm_matrix* m, hm_kernel_stat* out, int32_t nout);

/* hm_alg_bytes -- bytes the launches of one hm_matvec move per right-hand side
 * (the sum over its launches of the bytes hm_profile_read reports): the
 * method's bytes (hm_info_t.bytes_alg) plus the traffic of this layout's
 * intermediate steps (copy descriptors, per-piece input segments and multiplier
 * runs, segment partials, fan-out slots). */
hm_status hm_alg_bytes(const hm_matrix* m, int64_t* bytes);

/*
 * hm_decompress_debug -- decode packed values of m's resident payload on the
 * GPU with the decoders the product kernels run (Sec. 4.1, Alg. 8), for the
 * bit-exact check of decompression against the CPU oracle.
 *   tier : 0 = the FP32-tier decoders (column dots, row chunks and the
 *          multi-RHS kernels of matrices compressed at eps > 2^-22): tail = 0,
 *          head = the stored value rounded to nearest FP32 (ties to even) for
 *          codes of at most 24 significant bits (FPX e8, AFLP up to 3 bytes);
 *          wider codes are cut to FP32's 23 mantissa bits first (AFLP: s cut,
 *          then s - 1 rounded once), within 2^-22 + 2^-24 relative;
 *          1 = the float-float-tier decoders (eps <= 2^-22 and HM_CODEC_NONE):
 *          head + tail = the stored value (exact for every AFLP code with
 *          m' <= 47 and f <= 46 and every FPX code up to e11 m44; a raw FP64
 *          value keeps its low 29 mantissa bits rounded to 24, within 2^-48
 *          relative; AFLP codes beyond those limits within 2^-46 relative).
 *          Either tier may be asked for on any matrix.
 *   u0, u1 : units [u0, u1) (column-dot pieces 0 .. nitems-1, then row-chunk
 *          pieces; hm_info_t.nunits in all); u1 is clamped to nunits.
 *   Values come in payload order: unit by unit, column by column, row by row.
 *   AFLP values are +-(s - 1) with s = 2^f (1 + mant 2^-m'): the array's vmin
 *   is not applied (the kernels fold it into the coefficient and tile scales).
 *   head, tail : host float[cap]; code : host uint64[cap], each value's code
 *   (8 B bits, little-endian bytes of the payload); fmt : host uint16[cap], its
 *   format B | fmt << 4 | e << 6 | m << 10 (fmt 0 FPX e8, 1 FPX e11, 2 AFLP,
 *   3 raw FP64; m = m' for AFLP).  count : receives the number of values.
 *   With head == NULL only *count is set (no GPU work).
 * Allocates device memory for the call, synchronises `stream`.
 * Errors: HM_ERR_ARG (null count, bad tier or range, cap < count),
 * HM_ERR_STATE (not compressed), HM_ERR_OOM, HM_ERR_CUDA; an unknown decode
 * class latches HM_ERR_DEVICE (hm_sync_status).
 */
hm_status hm_decompress_debug(hm_matrix* m, int32_t tier, int64_t u0, int64_t u1, int64_t cap, float* head,
                              float* tail, uint64_t* code, uint16_t* fmt, int64_t* count, void* stream);

/*
 * Triangular solves with H-LU factors (Sec. 5, Conclusion: the triangular
 * solves of an H-LU factorisation read the same compressed blocks as the
 * product, with sequential dependencies).  x := U^-1 L^-1 b for A = L U without
 * pivoting (L unit lower, U upper triangular, cluster order): meant for
 * matrices whose unpivoted elimination is stable, such as the SPD Matern
 * covariance matrix.
 *
 * hm_lu_build -- host: dense elimination of the kernel matrix of prm on pts
 *   (cluster tree and block tree as hm_build; prm->format is not used), then
 *   the factors cut along A's block tree: a leaf block (t, s) with t after s
 *   goes to L, t before s to U, a diagonal leaf (t, t) holds the unit lower
 *   triangle of L_tt and the upper triangle of U_tt; admissible blocks are
 *   truncated at sigma_k <= prm->eps_build sigma_0 (eqn. epsilon), the others
 *   stay exact.  The dense array limits n to 8192.
 *   Errors: HM_ERR_ARG, HM_ERR_CAPACITY (n > 8192), HM_ERR_OOM,
 *   HM_ERR_UNSUPPORTED (a pivot vanished).
 * hm_lu_compress -- pack both factors as H-matrices (Sec. 4.1-4.2: direct
 *   compression of dense blocks and triangles, VALR columns of low-rank
 *   blocks) with eps / codec / valr as hm_compress, and upload them with the
 *   work list of the solve.  Synchronises the device.
 *   Errors: HM_ERR_ARG, HM_ERR_OOM, HM_ERR_CUDA, HM_ERR_UNSUPPORTED.
 * hm_lu_solve -- x := U^-1 L^-1 b for nrhs columns (device FP64, original
 *   point order, column-major, leading dimensions ldb, ldx >= n; x must not
 *   overlap b), stream-ordered, no sync.  Each column is one persistent
 *   cooperative launch: warps take the leaf solves (forward over the leaves,
 *   then backward) and the coefficient products t_b = S X^T z of the low-rank
 *   factor blocks in a dependency order, each waiting (bounded) for what it
 *   reads; values are decoded exactly (head + tail) and the arithmetic is FP64.
 *   A wait that runs out latches HM_ERR_TIMEOUT (hm_lu_sync_status).
 *   Errors: HM_ERR_ARG, HM_ERR_STATE (not compressed), HM_ERR_CUDA.
 * hm_lu_sync_status -- as hm_sync_status, for the solve's error word.
 * hm_lu_info -- stats[0 .. min(nstats, 7)) = n, packed payload bytes, packed
 *   code bytes, FP64 bytes of the same factors, work items, leaves, low-rank
 *   blocks.  Errors: HM_ERR_ARG.
 * hm_lu_free -- release host and device memory (NULL accepted).
 */
typedef struct hm_lu hm_lu;
hm_status hm_lu_build(const hm_build_params* prm, const double* pts, int64_t n, hm_lu** out);
hm_status hm_lu_compress(hm_lu* f, double eps, int32_t codec, int32_t valr);
hm_status hm_lu_solve(hm_lu* f, const double* b, int64_t ldb, double* x, int64_t ldx, int64_t nrhs, void* stream);
hm_status hm_lu_sync_status(hm_lu* f, void* stream);
hm_status hm_lu_info(const hm_lu* f, int64_t* stats, int32_t nstats);
hm_status hm_lu_free(hm_lu* f);

/*
 * hm_matvec_host_noalloc -- hm_matvec_host for callers that cannot let the
 * library allocate device memory.  (The paper has no counterpart: this is a
 * deployment aid.)  A serving process that has committed its whole HBM budget
 * up front, or code that must not trigger cudaFree's device-wide
 * synchronisation while other streams run, cannot use hm_matvec_host, which
 * allocates (and may re-allocate) its device staging buffers.  This entry
 * point stages x and y instead through one fixed array compiled into libhm
 * (2 * HM_NOALLOC_MAX_ENTRIES doubles, 16 MiB, held on every GPU that loads
 * the library until the process exits) and calls no cudaMalloc or cudaFree.
 *   m, alpha, beta, nrhs, stream : as hm_matvec_host (m must be compressed).
 *   x, y : host FP64 (n x nrhs, ld n, column-major); y is overwritten with
 *          alpha*M*x + beta*y.  Synchronises `stream` before returning.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life of
 * the process; make that first call before any stream capture.  The kept
 * address belongs to the device's primary context: after cudaDeviceReset (a new
 * primary context) it is stale, so do not call this entry point on a device
 * that was reset.  With lazy module loading (the CUDA default) the array's
 * memory is committed when the library's device code first loads on the
 * device, by the CUDA runtime, not by a cudaMalloc of this call.  All calls
 * share the one array, which keeps the last call's contents: calls whose GPU
 * work overlaps (other host threads, other streams) race and must be
 * serialised by the caller.  x is copied in whole on every call, and y too when
 * beta != 0; with beta == 0 the product writes every entry of y without
 * reading it, so no earlier contents are read and nothing needs clearing.
 * Errors: HM_ERR_ARG, HM_ERR_STATE (not compressed), HM_ERR_CAPACITY if
 * n * nrhs > HM_NOALLOC_MAX_ENTRIES, HM_ERR_CUDA.
 */
#define HM_NOALLOC_MAX_ENTRIES (1 << 20)
hm_status hm_matvec_host_noalloc(hm_matrix* m, double alpha, const double* x, double beta, double* y,
                                 int64_t nrhs, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HM_H */
