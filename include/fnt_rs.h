/*
 * fnt_rs.h -- C ABI of libfntrs.so: FNT-based Reed-Solomon erasure codes
 * over the Fermat prime field F_65537 on one GB300 GPU (sm_103a).
 *
 * Method: Soro & Lacan, "FNT-based Reed-Solomon Erasure Codes".
 *   - field and root of unity: Sec. II.A (3 is a primitive root of GF(65537))
 *     and Sec. II.B (r = 3^(2^(16-i)) has order n = 2^i);
 *   - non-systematic encoding e_i = s(r^i), i < n, by one FNT of the
 *     zero-padded source: Sec. II.B;
 *   - erasure decoding by interpolation, steps 1-6 of Sec. II.B: per erasure
 *     pattern A(x) = prod (x - x_i), A'(x_i); per codeword n_i = v_i / A'(x_i),
 *     the power series sum n_i / (x - x_i) by one FNT, and the product with A;
 *   - per-pattern work done once for many codewords: Sec. II.B (last part).
 *
 * Data layout (all buffers are owned by the caller; Sec. II.B interleaving):
 *   a batch of W codewords is a row-major matrix whose column c is codeword c.
 *     source   src[k][ld_src]   uint16  (row i = source symbol i / packet i)
 *     encoded  enc[n][ld_enc]   uint32  values in [0, 65536]
 *     received recv[npos][ld]   uint32  row i = symbols received at positions[i]
 *     decoded  out[k][ld_out]   uint16
 *   Leading dimensions are in elements, ld >= W.  Device pointers must be
 *   4-byte aligned for uint16 buffers when W is even, 4-byte aligned for
 *   uint32 buffers.
 *
 * Streams: every `stream` argument is a cudaStream_t passed as void*
 * (NULL = legacy default stream).  Calls enqueue work and return without
 * synchronising, except where noted.
 *
 * Empty batches: W = 0 is a valid batch of no codewords; its data pointers
 * may be NULL and nothing is launched (a decode still validates the
 * positions and builds or finds their pattern).
 *
 * Errors: every int-returning call returns FNT_RS_OK (0) or a negative
 * FNT_RS_E_* code; no exception crosses the ABI.  Argument errors are
 * detected on the host before any launch.  Data-dependent conditions found
 * on the device (a decoded coefficient equal to 65536, a received value above
 * 65536, a device wait that gave up) are ORed into a per-plan status word that
 * fnt_rs_status() reads and clears.
 *
 * Allocation: plan creation allocates the plan's device tables; encode,
 * decode and FNT calls never allocate -- their scratch is the caller's
 * `workspace` of fnt_rs_workspace_bytes() bytes (may be NULL when that size
 * is 0).  A decode with a new erasure pattern builds the pattern's tables into
 * plan-owned buffers reserved at plan creation.
 *
 * Thread safety: a plan may be used from one host thread at a time.
 */
#ifndef FNT_RS_H
#define FNT_RS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FNT_RS_P 65537u

enum fnt_rs_status_code {
  FNT_RS_OK = 0,
  FNT_RS_E_ARG = -1,            /* bad pointer, size, alignment or leading dimension */
  FNT_RS_E_UNSUPPORTED_P = -2,  /* p != 65537 */
  FNT_RS_E_ROOT = -3,           /* root does not have order exactly n */
  FNT_RS_E_POSITIONS = -4,      /* fewer than k positions, a duplicate, or one >= n */
  FNT_RS_E_BUDGET = -5,         /* admission refused: request exceeds the memory budget */
  FNT_RS_E_CUDA = -6,           /* a CUDA runtime call failed */
  FNT_RS_E_RANGE = -7,          /* status: decoded 65536 (written as 0) or received > 65536 */
  FNT_RS_E_TIMEOUT = -8,        /* status: a bounded device wait gave up */
  FNT_RS_E_WORKSPACE = -9,      /* workspace missing or too small */
  FNT_RS_E_BOUNDS = -10         /* status, debug build only: a device index check failed */
};

enum fnt_rs_op {
  FNT_RS_OP_ENCODE = 0,
  FNT_RS_OP_DECODE = 1,
  FNT_RS_OP_FNT = 2,
  FNT_RS_OP_ENCODE_HOST = 3,    /* fnt_rs_encode_host staging */
  FNT_RS_OP_DECODE_HOST = 4,    /* fnt_rs_decode_host staging */
  FNT_RS_OP_ENCODE_SYS = 5,     /* fnt_rs_encode_sys */
  FNT_RS_OP_DECODE_SYS = 6,     /* fnt_rs_decode_sys */
  FNT_RS_OP_ENCODE_WIRE = 7,    /* fnt_rs_encode_wire */
  FNT_RS_OP_DECODE_WIRE = 8,    /* fnt_rs_decode_wire */
  FNT_RS_OP_ENCODE_WIRE_HOST = 9,   /* fnt_rs_encode_wire_host staging */
  FNT_RS_OP_DECODE_WIRE_HOST = 10   /* fnt_rs_decode_wire_host staging */
};

typedef struct fnt_rs_plan_s* fnt_rs_plan;

/*
 * Create a plan for codes of length n and dimension k over F_p.
 *   n     : power of two, 2 <= n <= 65536 (Sec. II.B: n = 2^i, n < 65537)
 *   k     : 1 <= k <= n (Sec. II.B: k <= n; k need not be a power of two)
 *   p     : must be 65537, else FNT_RS_E_UNSUPPORTED_P
 *   root  : 0 selects the paper's r = 3^(65536/n) (Sec. II.B); any other value
 *           must have order exactly n, else FNT_RS_E_ROOT.  Other roots
 *           define other (still MDS) codes.
 *   stream: stream on which the plan's tables are uploaded.
 * On success *out owns device tables until fnt_rs_plan_destroy.
 */
int fnt_rs_plan_create(fnt_rs_plan* out, uint32_t n, uint32_t k, uint32_t p, uint32_t root,
                       void* stream);

/* Synchronises the device, then frees the plan and its device tables. NULL is a no-op. */
void fnt_rs_plan_destroy(fnt_rs_plan plan);

/* Bytes of device workspace a call of kind `op` (enum fnt_rs_op) needs for W codewords. */
size_t fnt_rs_workspace_bytes(fnt_rs_plan plan, size_t W, int op);

/*
 * Non-systematic encode (Sec. II.B): enc[j][c] = s_c(r^j) for j < n, c < W,
 * where s_c(x) = sum_{i<k} src[i][c] x^i.  Output values lie in [0, 65536].
 * src, enc: device pointers; workspace: device, fnt_rs_workspace_bytes(plan,
 * W, FNT_RS_OP_ENCODE) bytes.  Enqueued on `stream`.
 */
int fnt_rs_encode(fnt_rs_plan plan, const uint16_t* src, size_t ld_src, uint32_t* enc,
                  size_t ld_enc, size_t W, void* workspace, void* stream);

/*
 * Schedules: how an encode or a decode is laid out on the GPU.  Every
 * schedule computes the same words (the arithmetic is exact); they differ in
 * staging and in how the length-n transform is split over CTAs and passes:
 *   FNT_RS_SCHED_TMA    one CTA per tile of codewords, rows staged in shared
 *                       memory by TMA (n <= 8192; decode also k <= n/2),
 *   FNT_RS_SCHED_TILE   one CTA per tile, rows loaded directly (n <= 32768;
 *                       decode: n <= 16384, or n = 32768 with k <= n/2),
 *   FNT_RS_SCHED_SPLIT  radix-(n/4096) cross passes and 4096-point local
 *                       passes through the workspace (encode n > 8192,
 *                       decode n >= 16384),
 *   FNT_RS_SCHED_CPA    decode only: tiles staged by cp.async (k <= n/2):
 *                       half-width tiles, two CTAs per SM, for n = 4096 or
 *                       8192; the one-CTA tile's two (one) codewords for
 *                       n = 16384 (32768),
 *   FNT_RS_SCHED_PAPER  decode only: the paper's own route (Sec. II.B/III):
 *                       step 3 by the chirp (per pattern), step 5 as a
 *                       middle product and step 6 as a product, both by
 *                       FNT_2n -- 4 FNT_2n per codeword against the 3 FNT_n
 *                       of the other schedules; for comparison (n <= 32768,
 *                       k <= n/2, default root).  Selecting it builds its
 *                       tables (synchronising the device) and grows the
 *                       decode workspace by 2 * 2n * W * 4 bytes (query the
 *                       size after selecting it); the autotuner never picks it,
 *   FNT_RS_SCHED_DIRECT the quadratic method (Sec. III) as one matrix product
 *                       over F_p per batch on the tensor cores (k <= 1024,
 *                       n <= 16384, default root): encode by the n x k matrix
 *                       r^(ij); decode by the k x k matrix of the Lagrange
 *                       basis coefficients of the first k positions (built on
 *                       the host once per erasure pattern).  Selecting it
 *                       builds the plan-level matrix (synchronising the
 *                       device); the workspace covers it once selected.  A
 *                       16-bit wire encode (fnt_rs_encode_wire) keeps the
 *                       transform schedules.
 * FNT_RS_SCHED_AUTO (the default) takes TMA where it applies, else (decode
 * of n = 16384, k <= n/2) CPA, else TILE (encode up to n = 8192; decode
 * wherever one CTA holds the codeword), else SPLIT.  fnt_rs_workspace_bytes covers every schedule of the plan.
 */
enum fnt_rs_sched {
  FNT_RS_SCHED_AUTO = 0,
  FNT_RS_SCHED_TMA = 1,
  FNT_RS_SCHED_TILE = 2,
  FNT_RS_SCHED_SPLIT = 3,
  FNT_RS_SCHED_CPA = 4,
  FNT_RS_SCHED_PAPER = 5,
  FNT_RS_SCHED_DIRECT = 6
};

typedef struct fnt_rs_tune_result_s {
  int sched; /* enum fnt_rs_sched */
  float us;  /* median time of one call, microseconds */
} fnt_rs_tune_result;

/* Forces the schedule of `op` (FNT_RS_OP_ENCODE or FNT_RS_OP_DECODE);
 * FNT_RS_E_ARG if it cannot run this plan.  FNT_RS_SCHED_AUTO restores the
 * default choice.  For FNT_RS_OP_ENCODE_SYS / FNT_RS_OP_DECODE_SYS the
 * choices are FNT_RS_SCHED_AUTO (the FNT route) and FNT_RS_SCHED_DIRECT, the
 * paper's quadratic methods for short codes (Sec. III, Tables I-II): the
 * encoder computes the n_out - k non-systematic symbols as products by the
 * (n - k) x k matrix of the Lagrange basis of r^0..r^(k-1) evaluated at r^j
 * (built on the host when selected); the decoder copies the received source
 * symbols and computes each missing one as a product by the Lagrange basis of
 * the first k received positions at r^m (built on the host once per erasure
 * pattern, then uploaded on `stream`).  Neither needs a workspace; k <= 1024,
 * n <= 16384, default root; same results as the FNT route. */
int fnt_rs_set_schedule(fnt_rs_plan plan, int op, int sched);
/* The schedule `op` runs with now (never FNT_RS_SCHED_AUTO), or a negative error. */
int fnt_rs_get_schedule(fnt_rs_plan plan, int op);

/*
 * Autotuner.  Runs every transform schedule of `op` that can run this plan
 * (TMA, CPA, TILE, SPLIT: never FNT_RS_SCHED_PAPER or FNT_RS_SCHED_DIRECT, so
 * a tuned plan computes its encode and decode on the integer pipes only; the
 * tensor-core product runs only when selected by fnt_rs_set_schedule) on W
 * codewords of zeroed data (at most 2^29 bytes of encoded words: a larger W
 * is timed on fewer columns, a multiple of 8) in device buffers it allocates
 * and frees itself, times each with CUDA events on `stream` (median of 5
 * calls after 2 warm-up calls; the time of an integer transform does not
 * depend on the data), keeps the fastest for the plan and writes up to `cap`
 * {schedule, microseconds} entries to `out`.  A decode tune builds a pattern
 * of its own in the plan's pattern cache (which may evict a cached pattern).
 * Synchronises `stream`.  Returns the number of schedules timed, or a
 * negative error (the plan's previous choice is then kept).
 */
int fnt_rs_autotune(fnt_rs_plan plan, size_t W, int op, fnt_rs_tune_result* out, int cap,
                    void* stream);

/*
 * Per-pattern preparation, steps 1-3 of the interpolation (Sec. II.B):
 * from the first k of `positions` (host array, npos >= k entries, distinct,
 * each < n) build on the device A(x) = prod (x - r^z_i), the weights
 * -r^(-z_i) / A'(r^z_i) and the transform of A mod x^k used by step 6.
 * Cached per plan: a later decode with the same first k positions reuses it.
 * Enqueued on `stream`; the host array may be reused when the call returns.
 */
int fnt_rs_decode_prepare(fnt_rs_plan plan, const uint32_t* positions, uint32_t npos,
                          void* stream);

/*
 * Erasure decode (Sec. II.B, steps 4-6 per codeword; steps 1-3 through the
 * pattern cache): out[j][c], j < k, are the coefficients of the unique
 * polynomial of degree < k through (r^positions[i], recv[i][c]), i < k.
 * recv: device [npos][ld_recv] uint32 (rows beyond k are ignored);
 * positions: host; out: device [k][ld_out] uint16.  A coefficient equal to
 * 65536, which no 16-bit source symbol has, is written as 0 and raises
 * FNT_RS_E_RANGE in the status word, as does a received value above 65536.
 * With all n positions received this is the inverse FNT's first k outputs
 * (Sec. II.B).
 */
int fnt_rs_decode(fnt_rs_plan plan, const uint32_t* recv, size_t ld_recv,
                  const uint32_t* positions, uint32_t npos, uint16_t* out, size_t ld_out,
                  size_t W, void* workspace, void* stream);

/*
 * Lossless decode (Sec. II.B: with nothing lost, decoding is the product by
 * the inverse FNT matrix and the decoded symbols are its first k outputs):
 * out[j][c] = (n^-1 sum_i enc[i][c] r^(-ij)) for j < k, one inverse FNT per
 * codeword instead of the three transforms of the interpolation.  enc:
 * device [n][ld_enc] uint32 holding all n symbols in position order; out:
 * device [k][ld_out] uint16.  For a valid codeword this equals fnt_rs_decode
 * with any k positions; for other inputs it is the first k coefficients of
 * the degree < n interpolant.  A value 65536 is written as 0 and raises
 * FNT_RS_E_RANGE in the status word.  workspace: FNT_RS_OP_FNT bytes.
 */
int fnt_rs_decode_full(fnt_rs_plan plan, const uint32_t* enc, size_t ld_enc, uint16_t* out,
                       size_t ld_out, size_t W, void* workspace, void* stream);

/*
 * Erasure decode from a receiver's slot buffer (Sec. II.B, same steps as
 * fnt_rs_decode): slots is a device [n][ld_slots] uint32 matrix whose row z
 * holds the symbols received at position z (rows of erased positions are
 * never read).  Only the first k entries of `positions` are used.  Plans with
 * a non-default root return FNT_RS_E_ROOT (their positions are not slot rows).
 */
int fnt_rs_decode_slots(fnt_rs_plan plan, const uint32_t* slots, size_t ld_slots,
                        const uint32_t* positions, uint32_t npos, uint16_t* out, size_t ld_out,
                        size_t W, void* workspace, void* stream);

/*
 * Batched FNT of length n (Sec. II.A): out[j][c] = sum_i in[i][c] r^(ij)
 * (inverse = 0) or n^-1 sum_i in[i][c] r^(-ij) (inverse = 1), all mod p,
 * outputs in [0, 65536].  in, out: device [n][ld] uint32 with values in
 * [0, 2^32) taken mod p; in and out must not overlap.
 */
int fnt_rs_fnt(fnt_rs_plan plan, const uint32_t* in, size_t ld_in, uint32_t* out, size_t ld_out,
               size_t W, int inverse, void* workspace, void* stream);

/*
 * Host-buffer variants: same results as fnt_rs_encode / fnt_rs_decode with
 * host source and destination buffers (pinned memory gives asynchronous
 * copies).  Batches of W >= 1024 codewords are cut into up to 4 column
 * chunks whose host-to-device copies, kernels and device-to-host copies
 * overlap: the kernels run on `stream`, the copies on two streams the plan
 * owns, ordered after the work already queued on `stream`; the call
 * synchronises `stream` before returning, with every copy done.  workspace:
 * device, fnt_rs_workspace_bytes(plan, W, FNT_RS_OP_ENCODE_HOST /
 * FNT_RS_OP_DECODE_HOST) bytes; it also stages the data.  Host buffers are
 * dense (ld = W).  A plan's host-buffer calls must not run concurrently.
 */
int fnt_rs_encode_host(fnt_rs_plan plan, const uint16_t* h_src, uint32_t* h_enc, size_t W,
                       void* workspace, void* stream);
int fnt_rs_decode_host(fnt_rs_plan plan, const uint32_t* h_recv, const uint32_t* positions,
                       uint32_t npos, uint16_t* h_out, size_t W, void* workspace, void* stream);

/*
 * Encode without any allocation, scratch included (the paper has no
 * counterpart; this is a deployment convenience).  Codes with n > 8192 are
 * encoded in two passes that exchange data through n * W words of scratch, and
 * a punctured code is encoded at full length into n * W words first;
 * fnt_rs_encode takes that scratch from the caller, this call takes it from a
 * fixed device array of FNT_RS_NOALLOC_SCRATCH_BYTES that the library keeps on
 * every GPU it is loaded on until the process exits.  It is meant for callers
 * that cannot allocate device memory once they are running: services that
 * pre-reserve all device memory at start-up (or run inside a framework whose
 * allocator owns it) and so have no workspace to hand over, and latency-bound
 * pipelines that must not hit cudaMalloc's implicit device synchronisation or
 * an out-of-memory failure in the middle of a stream.
 *   - Same arguments and result as fnt_rs_encode, minus the workspace.
 *   - fnt_rs_workspace_bytes(plan, W, FNT_RS_OP_ENCODE) above
 *     FNT_RS_NOALLOC_SCRATCH_BYTES: returns FNT_RS_E_WORKSPACE without
 *     launching anything (split the batch into smaller W).  For an unpunctured
 *     code that size is n * W * 4 (capped by the column chunking); a punctured
 *     code with n > 8192 needs about twice that.
 *   - A code that needs no scratch (n <= 8192, not punctured) simply runs
 *     fnt_rs_encode.
 *   - The first call on a device looks up the array's device address; make
 *     that first call before any stream capture.
 *   - All calls share the one array: calls that overlap on the GPU race.
 */
#define FNT_RS_NOALLOC_SCRATCH_BYTES (16u << 20)
int fnt_rs_encode_noalloc(fnt_rs_plan plan, const uint16_t* src, size_t ld_src, uint32_t* enc,
                          size_t ld_enc, size_t W, void* stream);

/*
 * Punctured code (Sec. II.B: a length that is not a power of two is a
 * puncturing of the next power of two).  Keeps the first n_out positions of
 * the plan's length-n code, k <= n_out <= n: fnt_rs_encode and
 * fnt_rs_encode_sys then write n_out rows (the workspace grows by n * W * 4
 * bytes for the rows dropped), positions passed to the decoders must be below
 * n_out, and fnt_rs_decode_full (which needs every position) returns
 * FNT_RS_E_ARG.  n_out = n restores the full code.  FNT_RS_E_ARG if n_out is
 * out of range.
 */
int fnt_rs_plan_set_length(fnt_rs_plan plan, uint32_t n_out);

/*
 * Systematic code (the paper's "Toward a systematic code" section).  Encode:
 * the k source values of every codeword are interpolated at the first k
 * positions r^0..r^(k-1), which gives k intermediate symbols (coefficients of
 * a polynomial of degree < k over F_p); their length-n transform is the
 * codeword, whose first k rows are therefore the source itself.
 * src [k][ld_src] u16, enc [n_out][ld_enc] u32 (device).  Decode: the
 * intermediate symbols are interpolated from the first k of `positions` (as
 * fnt_rs_decode does) and transformed again; rows 0..k-1 of the result are
 * the source, written to out [k][ld_out] u16 (a value 65536 is written as 0
 * and raises FNT_RS_E_RANGE in the status word).  When the first k positions
 * are exactly 0, 1, ..., k-1 the decoder copies the received rows instead.
 * recv [npos][ld_recv] u32 (row i = positions[i]), positions on the host.
 * workspace: device, fnt_rs_workspace_bytes(plan, W, FNT_RS_OP_ENCODE_SYS /
 * FNT_RS_OP_DECODE_SYS) bytes (2 * n * W * 4 plus the decode's own); the
 * intermediate-symbol pattern is built on the first call (synchronising
 * `stream` once).  Default root only (FNT_RS_E_ROOT otherwise).  Enqueued on
 * `stream`.
 */
int fnt_rs_encode_sys(fnt_rs_plan plan, const uint16_t* src, size_t ld_src, uint32_t* enc,
                      size_t ld_enc, size_t W, void* workspace, void* stream);
int fnt_rs_decode_sys(fnt_rs_plan plan, const uint32_t* recv, size_t ld_recv,
                      const uint32_t* positions, uint32_t npos, uint16_t* out, size_t ld_out,
                      size_t W, void* workspace, void* stream);

/*
 * 16-bit wire format (Sec. II.B, "Design of the code on GF(65537)": every
 * symbol but 65536 fits in 16 bits; the positions that hold 65536 are sent
 * beside the packets, in their headers).  A symbol travels as its low 16
 * bits (65536 as 0) and every symbol equal to 65536 is listed as an escape
 * {row, col}: row = packet (encoded row, or index of a received row), col =
 * codeword.  On random data one symbol in 65537 is an escape.
 */
typedef struct fnt_rs_escape_s {
  uint32_t row, col;
} fnt_rs_escape;

/*
 * Encode to the wire format: the symbols of fnt_rs_encode, as 16 bits, into
 * enc [n_out][ld_enc] uint16 (device), and their escapes into esc (device,
 * esc_cap entries, in no particular order; each escaped symbol listed once).
 * *esc_count (device word) receives the number of escapes, also when it
 * exceeds esc_cap: the entries beyond esc_cap are then dropped (the symbols
 * are still complete) and the call can be repeated with a larger array.
 * fnt_rs_wire_escape_cap() is a capacity that random data never exceeds in
 * practice (about 1/64 of the symbols; the expected share is 1/65537); an
 * adversarial source can make up to k - 1 symbols of a codeword escapes.
 * workspace: fnt_rs_workspace_bytes(plan, W, FNT_RS_OP_ENCODE_WIRE) bytes (a
 * punctured code needs no extra rows: rows >= n_out are never stored).
 * esc must be 8-byte aligned, esc_count 4-byte aligned.  Enqueued on `stream`.
 */
size_t fnt_rs_wire_escape_cap(fnt_rs_plan plan, size_t W);
int fnt_rs_encode_wire(fnt_rs_plan plan, const uint16_t* src, size_t ld_src, uint16_t* enc,
                       size_t ld_enc, size_t W, fnt_rs_escape* esc, uint32_t esc_cap,
                       uint32_t* esc_count, void* workspace, void* stream);

/*
 * Decode from the wire format: recv [npos][ld_recv] uint16 (device, row i =
 * the packet received at positions[i]) and its escapes esc (device, nesc
 * entries, row = index of the received row, any order); otherwise as
 * fnt_rs_decode.  Escapes of rows >= k (not used by the decode) are skipped;
 * an escape outside the received rows or columns, or whose 16-bit symbol is
 * not 0, is not valid wire data: it raises FNT_RS_E_RANGE in the status word
 * (and the decoded words are then unspecified).  workspace:
 * fnt_rs_workspace_bytes(plan, W, FNT_RS_OP_DECODE_WIRE) bytes (the k rows
 * are widened to 32 bits there).  Enqueued on `stream`.
 */
int fnt_rs_decode_wire(fnt_rs_plan plan, const uint16_t* recv, size_t ld_recv,
                       const uint32_t* positions, uint32_t npos, const fnt_rs_escape* esc,
                       uint32_t nesc, uint16_t* out, size_t ld_out, size_t W, void* workspace,
                       void* stream);

/*
 * Host-buffer variants of the wire calls (dense host buffers, ld = W;
 * chunked and synchronised like fnt_rs_encode_host / fnt_rs_decode_host).  Encode: h_enc [n_out][W] uint16; the
 * escapes are written to h_esc sorted by row, then column, and their number
 * to *nesc.  Returns FNT_RS_E_ARG if they do not fit in esc_cap (*nesc then
 * says how many there are) and FNT_RS_E_WORKSPACE if they exceed
 * fnt_rs_wire_escape_cap(plan, W), the number the workspace stages (use
 * fnt_rs_encode_wire with a larger array).  Decode: h_recv [npos][W] uint16,
 * only its first k rows are copied; h_esc: nesc escapes (host).  workspace:
 * FNT_RS_OP_ENCODE_WIRE_HOST / FNT_RS_OP_DECODE_WIRE_HOST bytes.
 */
int fnt_rs_encode_wire_host(fnt_rs_plan plan, const uint16_t* h_src, uint16_t* h_enc, size_t W,
                            fnt_rs_escape* h_esc, uint32_t esc_cap, uint32_t* nesc,
                            void* workspace, void* stream);
int fnt_rs_decode_wire_host(fnt_rs_plan plan, const uint16_t* h_recv, const uint32_t* positions,
                            uint32_t npos, const fnt_rs_escape* h_esc, uint32_t nesc,
                            uint16_t* h_out, size_t W, void* workspace, void* stream);

/*
 * Reads the plan's device status word (synchronising `stream`), clears it and
 * returns FNT_RS_OK, FNT_RS_E_RANGE, FNT_RS_E_BOUNDS (debug build) or
 * FNT_RS_E_TIMEOUT (the most severe seen).
 */
int fnt_rs_status(fnt_rs_plan plan, void* stream);

/*
 * 1 if this library is the debug build (not part of the paper's method; a
 * development aid): every shared-memory index of the transform passes and
 * every global index of the loaders, storers and staged tiles is checked on
 * the device, and a failed check skips the access and raises FNT_RS_E_BOUNDS
 * in the status word instead of faulting.  0 in the release build, where the
 * checks are compiled out.
 */
int fnt_rs_debug_bounds(void);

/*
 * Ragged batches (many codeword groups of different n, k, W and erasure
 * pattern in one launch).  Each group is one round trip of the method:
 * encode src -> enc (Sec. II.B), build the group's pattern tables from the
 * first k of `positions` (steps 1-3), decode every codeword from enc used as
 * the receiver's slot buffer (row z = position z, steps 4-6) into out.
 * Groups with positions == NULL are encode-only.  All pointers are device
 * pointers except `positions` (host, copied at creation).  The library owns
 * one plan per distinct (n, k), each decode group's pattern tables and the
 * split-transform workspace; creation runs the batch once (uncaptured) and
 * captures it into one CUDA graph.  In that graph every group with
 * 256 <= n <= 8192 runs inside one launch of a persistent kernel (its CTAs
 * take the groups' encode tiles, pattern builds and decode tiles from one
 * work list); the other groups keep per-group launches spread over up to
 * `nstreams` streams, their plans' schedules picked by fnt_rs_autotune on the
 * widest group of each plan (environment FNTRS_AUTOTUNE=0 keeps the default
 * schedules).  Groups must not share output buffers.
 * Failure-detection test hook: with the environment variable
 * FNTRS_TEST_STALL_GROUP=g at creation, the decode items of persistent group
 * g wait for one encode tile more than the group has (a stalled producer);
 * their bounded waits give up, FNT_RS_E_TIMEOUT is raised in the status word
 * and that group's decode is skipped, everything else completes.
 */
typedef struct fnt_rs_group_s {
  uint32_t n, k;
  size_t W;
  const uint16_t* src;
  size_t ld_src;
  uint32_t* enc;
  size_t ld_enc;
  const uint32_t* positions; /* host, npos >= k entries; NULL: encode only */
  uint32_t npos;
  uint16_t* out;
  size_t ld_out;
} fnt_rs_group;

typedef struct fnt_rs_ragged_s* fnt_rs_ragged;

int fnt_rs_ragged_create(fnt_rs_ragged* out, const fnt_rs_group* groups, uint32_t ngroups,
                         uint32_t nstreams, void* stream);
/* Replays the captured graph on `stream` (one graph launch, no host sync). */
int fnt_rs_ragged_run(fnt_rs_ragged r, void* stream);
/* The same work as plain per-group calls on `stream`, one after another (baseline). */
int fnt_rs_ragged_run_plain(fnt_rs_ragged r, void* stream);
/* ORs the status words of the batch's plans (synchronises `stream`). */
int fnt_rs_ragged_status(fnt_rs_ragged r, void* stream);
/* {groups, plans, streams, groups in the persistent kernel, its work items,
 * plans whose schedules were autotuned}; returns the number of ints written
 * (at most cap). */
int fnt_rs_ragged_info(fnt_rs_ragged r, int* info, int cap);
void fnt_rs_ragged_destroy(fnt_rs_ragged r);

/*
 * Serving loop (continuous batching).  A dispatcher thread admits requests
 * in arrival order as stream slots and device memory free up: each request's
 * input and output live in an arena of `budget_bytes` reserved at creation
 * (the admission budget); requests that arrive while others run start on
 * their own streams and overlap with them.  Plans, twiddle tables and the
 * per-pattern locator tables (steps 1-3, Sec. II.B; an LRU pool per plan)
 * stay resident.  A request's input is generated on the device from `seed`:
 * uniform 16-bit source symbols (encode, [k][W]) or uniform values in
 * [0, 65536] received at `positions` (decode, [k][W]).
 */
typedef struct fnt_rs_request_s {
  int op; /* FNT_RS_OP_ENCODE or FNT_RS_OP_DECODE */
  uint32_t n, k, W;
  uint64_t seed;
  const uint32_t* positions; /* decode: host, >= k entries, copied at submit */
  uint32_t npos;
} fnt_rs_request;

typedef struct fnt_rs_server_s* fnt_rs_server;

/* keep_results = 0 frees a request's buffers as soon as it completes. */
int fnt_rs_server_create(fnt_rs_server* out, size_t budget_bytes, uint32_t nstreams,
                         int keep_results);
/* Creates the plan of (n, k) now instead of at its first request. */
int fnt_rs_server_preplan(fnt_rs_server s, uint32_t n, uint32_t k);
/* Queues a request; FNT_RS_E_BUDGET if its buffers alone exceed the budget. */
int fnt_rs_server_submit(fnt_rs_server s, const fnt_rs_request* req, uint64_t* ticket);
/* 1 done (latency in *latency_ms), 0 queued or running, negative: its error. */
int fnt_rs_server_poll(fnt_rs_server s, uint64_t ticket, double* latency_ms);
/* Blocks until every submitted request has finished. */
int fnt_rs_server_drain(fnt_rs_server s);
/* Copies a finished request's input / output (kept results) to host memory. */
int fnt_rs_server_fetch(fnt_rs_server s, uint64_t ticket, void* h_in, void* h_out);
/* Frees a finished request's buffers and record. */
int fnt_rs_server_release(fnt_rs_server s, uint64_t ticket);
/* {completed, rejected, arena bytes in use, arena bytes, resident plans}. */
int fnt_rs_server_stats(fnt_rs_server s, double* out, int cap);
void fnt_rs_server_destroy(fnt_rs_server s);
/* Submits reqs[i] once arrival_s[i] seconds (real time) have passed since the
 * replay's start t0 and records latency_ms[i] counted from that due time
 * t0 + arrival_s[i] to the moment the dispatcher sees the result (queueing
 * and a late submission included; -1: refused); *wall_s = duration of the
 * replay.  fnt_rs_server_poll's latency counts from the submit call. */
int fnt_rs_server_replay(fnt_rs_server s, const fnt_rs_request* reqs, const double* arrival_s,
                         uint32_t count, double* latency_ms, double* wall_s);
/* Same trace through the plain path: one request at a time, its plan and
 * pattern built per request, on `stream`; latency on the same clock (due
 * time to result). */
int fnt_rs_baseline_replay(const fnt_rs_request* reqs, const double* arrival_s, uint32_t count,
                           double* latency_ms, double* wall_s, void* stream);

/* Static description of a status code. */
const char* fnt_rs_strerror(int code);

/* Number of kernel launches the library has issued since load (all plans). */
uint64_t fnt_rs_launch_count(void);

/*
 * Plan introspection for tuning and tests: writes up to `cap` ints
 * {n, k, L, C, Wt_encode, Wt_decode, schedule_id, pattern_cache_entries}.
 * Returns the number written.
 */
int fnt_rs_plan_info(fnt_rs_plan plan, int* info, int cap);

#ifdef __cplusplus
}
#endif

#endif /* FNT_RS_H */
