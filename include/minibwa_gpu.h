/*
 * minibwa_gpu: the seeding stage of minibwa (arxiv 2606.15357) on one GB300 GPU.
 *
 * For every read it finds the (l,c)-SMEMs against an FMD-index of the reference
 * (Section 2.1 definitions; Algorithm 3), flags SMEMs that occur more than
 * max_occ times, and locates the remaining occurrences through a sampled
 * suffix array by LF-walks (Section 2.4; Algorithm 2).  All arithmetic runs in
 * CUDA kernels for sm_103a; the host code below only moves data and launches.
 *
 * Conventions shared by every call:
 *  - Base codes: 0=A 1=C 2=G 3=T; 4 (or any value > 3) = N.
 *  - Pointers marked "host or device" are classified with
 *    cudaPointerGetAttributes; host buffers are staged through the library.
 *    The caller owns every buffer it passes in.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    enqueue work on it and return after the results they report on the host
 *    (counts, status) are known; device outputs are complete when they return.
 *  - Return value: MB_OK (0) or a negative MB_ERR_* code; mb_strerror() names
 *    it.  No C++ exception crosses this boundary.
 *  - An index is read-only after it is built and may be used from several
 *    streams at once.  A server (mb_serve_*) is used from one host thread.
 *  - Text coordinates: T = R . revcomp(R) . $ (Section 2.1), n = 2|R| + 1; in
 *    bisulfite mode R is replaced by CT(R) . GA(R) (Section 2.9).  n must be
 *    below 2^32.
 */
#ifndef MINIBWA_GPU_H
#define MINIBWA_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MB_OK = 0,
    MB_ERR_ARG = -1,          /* invalid argument (null pointer, size out of range, n >= 2^32) */
    MB_ERR_NOMEM = -2,        /* device or host allocation failed / admission budget exceeded */
    MB_ERR_CAPACITY = -3,     /* output buffer too small; the needed size is reported */
    MB_ERR_CUDA = -4,         /* a CUDA runtime call failed */
    MB_ERR_TIMEOUT = -5,      /* a bounded wait expired */
    MB_ERR_IO = -6,           /* file could not be opened, read or written */
    MB_ERR_CORRUPT = -7,      /* index file header or checksum mismatch */
    MB_ERR_DEVICE_CHECK = -8, /* a device-side consistency check failed */
    MB_ERR_BUSY = -9          /* server has no free slot for the request right now */
};

/* Flags of mb_opts.flags */
#define MB_BS3      0x1u   /* index: bisulfite 3-base index over CT(R).GA(R) (Section 2.9);
                              seeding: convert read 1 C->T and read 2 G->A, keep hits by strand */
#define MB_BATCHED  0x2u   /* seeding: lanes take reads from a device work queue, in read order */
#define MB_CHECKED  0x4u   /* seeding / locate: the kernels also check every occurrence row they
                              read against the text length (only a damaged index can fail it; the
                              checked locate runs one walk per lane); a failed check ends that read
                              or walk and the call returns MB_ERR_DEVICE_CHECK.  Without the flag the kernels still check every
                              read's offsets and every record's rows (MB_ERR_DEVICE_CHECK), and the
                              host checks every device buffer against its allocation (MB_ERR_ARG) */
#define MB_NO_KMER  0x8u   /* seeding: do not use the k-mer ds-interval table */
#define MB_COUNT    0x10u  /* seeding/locate: also count the work done (mb_work_counters) */
#define MB_NO_AUX   0x20u  /* index: build without the packed text and the rate-4 SA / ISA samples
                              (2.25 bytes per text position) that let seeding extend unique matches
                              by comparing text */
#define MB_STEP_ONLY 0x40u /* seeding: extend every match step by step (Algorithm 1), even where
                              the auxiliary arrays allow comparing text */
#define MB_LOCATE_JOIN 0x100u /* locate: the walked rows go in 8 passes (by a hash of the row); a walk
                              stops where it meets a walked row of an earlier pass and takes that
                              row's position plus its distance (same positions, fewer LF steps; 36
                              bytes per 64 index rows plus 4 bytes per walked row of device
                              workspace).  Off under MB_CHECKED.  By default every LF-walk runs to
                              its sampled row */
#define MB_LOCATE_AUX 0x200u /* locate: walks stop at the rate-4 SA samples the index keeps for
                              extending unique matches (a row that is a multiple of 4) instead of
                              the rate-r samples of Section 2.4: about r/4 times fewer LF steps, same
                              positions; no joins.  Ignored for an index built with MB_NO_AUX */
#define MB_SMEM_ONE_LOOP 0x80u /* tuning: the SMEM kernel in its one-loop form (every iteration runs
                              every stage's code) instead of the split form (uniform block steps,
                              the other actions in service passes); same output */

/* Flags of mb_smem.flags */
#define MB_SMEM_OVER_MAX_OCC 0x1u   /* s > max_occ: reported, not located, no hits */
#define MB_SMEM_ROUND2       0x2u   /* found by the second seeding round (mb_reseed) */

typedef struct mb_index mb_index;
typedef struct mb_server mb_server;

/* Parameters.  Zero in any field selects its default. */
typedef struct {
    uint32_t min_len;         /* l, minimum SMEM length (default 19, Section 2.6) */
    uint32_t min_occ;         /* c, minimum occurrence (default 1) */
    uint32_t max_occ;         /* SMEMs with s > max_occ are flagged and not located (default 500) */
    uint32_t sa_rate;         /* r, suffix array sample rate (default 32, Section 2.4) */
    uint32_t kmer_k;          /* k of the k-mer ds-interval table (default 10, Section 2.5), <= 16;
                                 the table takes 12 * 4^k bytes (3.2 GB at k = 14, 51.5 GB at
                                 k = 16) */
    uint32_t flags;           /* MB_* flags above */
    uint32_t chunk_reads;     /* mb_seed_locate: reads per pipelined chunk (0 = 2^22) */
    uint32_t prefetch_depth;  /* tuning: LF-walks in flight per lane in locate, 1/2/4/8/16 (0 = 1) */
    uint32_t block_size;      /* tuning: threads per block (0 = default) */
    uint32_t smem_burst;      /* tuning: SMEM kernel (split form), memory steps (extensions, walk
                                 steps, text comparisons, samples, k-mer entries) a warp runs between
                                 two service passes of its stage changes (0 = default, 8) */
    uint32_t smem_wait;       /* tuning: SMEM kernel (split form), lanes out of the memory steps that
                                 call a service pass early, 1..32 (0 = default, 8) */
    uint32_t smem_warps;      /* tuning: SMEM kernel (split form), resident warps per SM its register
                                 budget aims at: 40 (256 threads per block) or 48 (256 or 512); 0 =
                                 24 at 128 threads per block, else 32 */
    uint32_t smem_reads_per_warp; /* tuning: SMEM kernel (split form), reads a warp holds at once,
                                 one per lane, 1..32 (0 = 32); with fewer the other lanes stay idle
                                 (a read's steps depend on each other, so lanes cannot share one) */
} mb_opts;

/* One SMEM (48 bytes).  (k, kr, s) is its ds-interval (lo(P), lo(revcomp P), occ(P)),
 * P = read[qbeg, qend).  hit_off indexes its first hit in mb_locate's output. */
typedef struct {
    uint32_t read, qbeg, qend, flags;
    uint64_t k, kr, s;
    uint64_t hit_off;
} mb_smem;

/* ---------------------------------------------------------------------------------------
 * mb_index_build — FMD-index of a reference on the GPU (Section 2.1, 2.2, 2.3, 2.5).
 *   ref      host or device, `len` base codes; codes > 3 (ambiguous) are replaced by
 *            random bases: bits 63..62 of splitmix64's output function of
 *            (n_seed + (pos+1) * 0x9E3779B97F4A7C15)  (Section 2.1, "random bases").
 *   opts     sa_rate, kmer_k, flags & MB_BS3 are used.
 *   stream   stream for the build.
 *   out      receives the new index (free with mb_index_free).
 * Builds T, its suffix array by prefix doubling, the BWT in occurrence blocks (Section 2.2;
 * here 32 bytes per 64 rows: four u32 counts of A/C/G/T before the block, then the 64 2-bit
 * symbols as two bit planes), the sampled suffix array and the k-mer ds-interval table.
 * Errors: MB_ERR_ARG (len = 0, n >= 2^32), MB_ERR_NOMEM, MB_ERR_CUDA.
 */
int mb_index_build(const uint8_t *ref, uint64_t len, const mb_opts *opts, uint64_t n_seed,
                   void *stream, mb_index **out);

/* Write / read an index file (header with version, sizes and a checksum; the blocks as in
 * memory).  Errors: MB_ERR_IO, MB_ERR_CORRUPT (bad header, size or checksum, or auxiliary samples
 * at another rate than this library's), MB_ERR_NOMEM, MB_ERR_CUDA. */
int mb_index_save(const mb_index *idx, const char *path);
int mb_index_load(const char *path, void *stream, mb_index **out);
void mb_index_free(mb_index *idx);

/* n = |T|, primary = the row i with S(i) = 0, ref_len = |R| (|R3| in bisulfite mode). */
int mb_index_info(const mb_index *idx, uint64_t *n, uint64_t *primary, uint64_t *ref_len);

/* Copy index arrays to the caller (host or device): sa (n x u32, full suffix array; only
 * available until mb_index_drop_sa, else MB_ERR_ARG), bwt (n bytes, 0=$ 1..4=A..T),
 * ssa (ceil(n/r) x u32), occ blocks (n/64 + 1 blocks of 32 bytes: four u32 counts of A,C,G,T
 * before the block, then two u64 bit planes of its 64 rows: bit q of the first is the low bit of
 * row q's code 0..3, bit q of the second its high bit; the $ row reads as A), kmer table (4^k x 3 u32:
 * k, kr, s of the k-mer whose base t is in bits 2t..2t+1 of the entry number), C (5 x u64 =
 * #{B[i] < a} for a = $,A,C,G,T).  Any pointer may be NULL. */
int mb_index_export(const mb_index *idx, uint32_t *sa, uint8_t *bwt, uint32_t *ssa,
                    void *occ_blocks, uint32_t *kmer, uint64_t *C);
/* The auxiliary arrays of an index built without MB_NO_AUX (else MB_ERR_ARG when any pointer is
 * given): text2 ((n - 1 + 15) / 16 + 2 u32: T[0, n-1) at 2 bits per base, base e of word w in
 * bits 2e..2e+1, zero padding), sa_aux (ceil(n / 4) u32: S(4x)), isa_aux (ceil(n / 4) u32: the
 * row of the suffix at text position 4p).  No counterpart in the paper: they let seeding extend
 * a match that occurs once by comparing the read with the text (same SMEMs). */
int mb_index_export_aux(const mb_index *idx, uint32_t *text2, uint32_t *sa_aux, uint32_t *isa_aux);
/* Entries of the k-mer table (Section 2.5) for `n` k-mer codes (host array `codes`, each below
 * 4^k, base t of the k-mer in bits 2t..2t+1): out (host, 3n u32) receives (k, kr, s) per code, the
 * ds-interval of the k-mer.  Reads n x 12 bytes of the table instead of copying all of it (51.5 GB
 * at k = 16).  MB_ERR_ARG for a null pointer or a code of 4^k or more (nothing written). */
int mb_index_kmer_get(const mb_index *idx, const uint64_t *codes, uint64_t n, uint32_t *out);
/* Free the full suffix array kept after the build (it is only needed for mb_index_export). */
int mb_index_drop_sa(mb_index *idx);

/* ---------------------------------------------------------------------------------------
 * mb_seed_batch — (l,c)-SMEMs of a batch of reads (Section 2.5, Algorithm 3) with the
 * max-occurrence flag and hit offsets.
 *   seq      host or device, concatenated read base codes.
 *   off      host or device, n_reads + 1 u64 offsets into seq (read r = seq[off[r], off[r+1])).
 *   mate     host or device or NULL; per read 0 = single, 1 = read 1, 2 = read 2 (used with
 *            MB_BS3 to convert read 1 C->T and read 2 G->A before seeding, Section 2.9).
 *   out      host or device, room for `cap` records.  Records are ordered by read, then by
 *            ascending qbeg; s > max_occ sets MB_SMEM_OVER_MAX_OCC; hit_off is the
 *            exclusive prefix sum of s over records without that flag.
 *   n_out    receives the number of SMEMs.  If it exceeds cap, nothing is written to out and
 *            MB_ERR_CAPACITY is returned with *n_out = the needed count.
 *   n_hits   (may be NULL) receives the total number of hits to locate.
 * Errors: MB_ERR_ARG, MB_ERR_CAPACITY, MB_ERR_NOMEM, MB_ERR_CUDA, MB_ERR_DEVICE_CHECK.
 */
int mb_seed_batch(const mb_index *idx, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                  const uint8_t *mate, const mb_opts *opts, void *stream,
                  mb_smem *out, uint64_t cap, uint64_t *n_out, uint64_t *n_hits);

/* ---------------------------------------------------------------------------------------
 * mb_reseed — the second seeding round of Section 2.6.  For every record of `smem` (the first
 * round's (l,c)-SMEMs of the same reads, as mb_seed_batch wrote them) with qend - qbeg >= 2l and
 * s <= 10 and no MB_SMEM_OVER_MAX_OCC, finds the (floor((qend-qbeg)/2), s+1)-SMEMs of the
 * substring read[qbeg, qend) (the paper prints the length as floor((j-1)/2); read here as the
 * window length j - i).  Records are in read coordinates, flagged MB_SMEM_ROUND2, ordered by
 * their window (the order of `smem`) then by qbeg, with the max-occ flag and hit offsets of
 * mb_seed_batch (relative to this output; pass it to mb_locate for the hits).
 *   seq, off, mate: as for mb_seed_batch (host or device).  smem: host or device.
 *   Capacity and errors as mb_seed_batch.
 */
int mb_reseed(const mb_index *idx, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
              const uint8_t *mate, const mb_smem *smem, uint64_t n_smem, const mb_opts *opts,
              void *stream, mb_smem *out, uint64_t cap, uint64_t *n_out, uint64_t *n_hits);

/* ---------------------------------------------------------------------------------------
 * mb_seed_batch_noalloc — mb_seed_batch for callers that cannot allocate device memory.
 * The paper has no counterpart: this is an interface of this library only.  Some callers
 * cannot call cudaMalloc: a process whose device memory is reserved in full by another
 * allocator (a framework's caching allocator, a serving runtime that pre-reserves HBM), or a
 * latency-critical caller for which an allocation, which may synchronize the device, is not
 * acceptable.  This entry point allocates nothing: its scratch is a fixed 64 MiB device array
 * inside the library (every GPU that loads the library holds it until the process exits).
 *   seq, off, mate (or NULL) and out must be DEVICE pointers; the other arguments, the results
 *   and the errors are those of mb_seed_batch (same records, same order).
 *   A batch whose scratch need exceeds 64 MiB (about 145,000 reads of 150 bases, less with many
 *   SMEMs) is rejected with MB_ERR_ARG and a message naming the need; split the batch.
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress) for
 *   that device and keeps it for later calls; make that first call before any stream capture.
 *   The kept address belongs to the device's current context: after cudaDeviceReset on that
 *   device it is stale, so do not call this entry point again in that process after a reset.
 *   All calls share the one array and it keeps the last call's contents: calls whose work
 *   overlaps on the GPU (from other streams or host threads) race and must not be issued;
 *   calls on one stream are ordered.
 */
int mb_seed_batch_noalloc(const mb_index *idx, const uint8_t *seq, const uint64_t *off,
                          uint32_t n_reads, const uint8_t *mate, const mb_opts *opts, void *stream,
                          mb_smem *out, uint64_t cap, uint64_t *n_out, uint64_t *n_hits);

/* ---------------------------------------------------------------------------------------
 * mb_locate — text positions of every row of every SMEM without MB_SMEM_OVER_MAX_OCC
 * (Section 2.4, Algorithm 2): row x is LF-walked to a sampled row; its position is
 * (steps + S(sampled row)) mod n.
 *   smem     host or device, n_smem records from mb_seed_batch (hit_off must be as written).
 *   hits     host or device, room for `cap` u32 positions; hit t of record m is written at
 *            hits[m.hit_off + t], rows k..k+s-1 in order.
 *   n_hits   receives the total.  If it exceeds cap: MB_ERR_CAPACITY, nothing written.
 * With MB_BS3 in opts, hits are still all written; mb_bs_filter applies the strand rule.
 * A row that several records share (the same or nested intervals) is walked once and its
 * position copied to each of their hits; with MB_COUNT the work counters count those walks.
 * Device workspace: about 40 bytes per record and 8 per hit, allocated per call.
 */
int mb_locate(const mb_index *idx, const mb_smem *smem, uint64_t n_smem, const mb_opts *opts,
              void *stream, uint32_t *hits, uint64_t cap, uint64_t *n_hits);

/* ---------------------------------------------------------------------------------------
 * mb_seed_locate — the whole stage in one call: SMEMs as mb_seed_batch, then their hits as
 * mb_locate (Section 2.5, Algorithm 3; Section 2.4, Algorithm 2), for callers whose reads and
 * results live in host memory.  The batch is cut into slices (at most 2^25 reads and 2^33
 * bases) and a slice into chunks of consecutive reads (opts->chunk_reads reads, at most 2^29
 * bases, at least one read) that alternate between two internal streams, so that the copies of
 * one chunk overlap the seeding of the other; each slice is then located at once (its repeated
 * rows walked once) while its records are copied out.  Use pinned host buffers for the copies
 * to overlap.  The environment variable MB_SLICE_READS, when set below 2^25, lowers the reads
 * per slice (less device memory, fewer repeated rows shared).
 *   seq, off, mate   host or device, as for mb_seed_batch.
 *   out              host or device, room for `cap` records: the records of mb_seed_batch (read
 *                    numbers and hit_off relative to this batch).
 *   hits             host or device, room for `hits_cap` u32: the output of mb_locate.
 *   n_out, n_hits    receive the totals.  If either exceeds its capacity, MB_ERR_CAPACITY is
 *                    returned with both totals; the contents of out and hits are then undefined.
 * Work is ordered after what the caller enqueued on `stream` before the call; the call returns
 * when every result is written.  Its device workspace (two seeding plans sized for the largest
 * chunk, two streams, staging buffers) is allocated on first use and kept for later calls with
 * the same index, device and seeding options whose chunks fit it (at most two such sets are
 * kept; mb_index_free releases them), so repeated calls allocate nothing.  Calls from several
 * host threads are allowed: each takes its own workspace.  A chunk that yields more records or
 * hits than its plan holds is seeded again through the allocating path.
 * Errors: MB_ERR_ARG, MB_ERR_CAPACITY, MB_ERR_NOMEM, MB_ERR_CUDA, MB_ERR_DEVICE_CHECK.
 */
int mb_seed_locate(const mb_index *idx, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                   const uint8_t *mate, const mb_opts *opts, void *stream, mb_smem *out, uint64_t cap,
                   uint32_t *hits, uint64_t hits_cap, uint64_t *n_out, uint64_t *n_hits);

/* ---------------------------------------------------------------------------------------
 * Batched form: a reusable seeding plan.
 * mb_plan_create allocates, once, all device workspace for batches of at most max_reads reads
 * and max_bases bases yielding at most max_smem SMEMs and max_hits hits.  mb_plan_run enqueues
 * the whole stage on `stream` (SMEMs by Algorithm 3, the max-occ flag, hit offsets, locate by
 * Algorithm 2) with no host synchronization and no allocation, so the call can be captured into
 * a CUDA graph and the graph replayed for new batches written into the same input buffers.
 * With MB_BATCHED in opts->flags the SMEM kernel takes reads from a device work queue in read
 * order (one persistent launch for reads of very different lengths: a lane takes the next read
 * when its read ends);
 * opts->block_size (128, 256 or 512) selects the launch shape.
 *   seq, off, mate (or NULL): DEVICE pointers, as in mb_seed_batch.
 * mb_plan_result waits for the stream and returns the plan-owned DEVICE arrays of the last
 * run (valid until the next run): records as mb_seed_batch writes them, and hits as mb_locate
 * writes them.  MB_ERR_CAPACITY (with the needed counts in *n_smem / *n_hits) if a limit was
 * exceeded; nothing beyond the limits was written.
 * mb_autotune times mb_plan_run on the given batch over the launch shapes in two stages and
 * writes the fastest into *best (same output for all): first the SMEM kernel's shape, threads per
 * block 128/256/512 x work queue off/on x kernel form (the one-loop form MB_SMEM_ONE_LOOP, or the
 * split form with smem_burst 2/4/8/16 x smem_wait 4/8/16), with 16 plain locate walks per lane;
 * then, when the best is a split form, smem_reads_per_warp 1/2/4/8/16 (against its 32); then, with
 * the best SMEM shape, locate walks per lane 1/2/4/8 plain and 1/2/4/8/16 with walks that join
 * (MB_LOCATE_JOIN) (92 points, 87 when the one-loop form wins).  mb_autotune_points does
 * the same and also returns every point tried with its time in ms (up to cap points; *n_points
 * receives the number tried).
 */
typedef struct mb_plan mb_plan;
int mb_plan_create(const mb_index *idx, const mb_opts *opts, uint32_t max_reads, uint64_t max_bases,
                   uint64_t max_smem, uint64_t max_hits, mb_plan **out);
int mb_plan_run(mb_plan *plan, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                const uint8_t *mate, void *stream);
int mb_plan_result(mb_plan *plan, void *stream, const mb_smem **smem, uint64_t *n_smem,
                   const uint32_t **hits, uint64_t *n_hits);
void mb_plan_free(mb_plan *plan);
/* Copy the last run's records / hits (counts from mb_plan_result) into caller buffers, host or
 * device; either pointer may be NULL.  MB_ERR_CAPACITY if a buffer is too small. */
int mb_plan_copy(mb_plan *plan, void *stream, mb_smem *out, uint64_t cap, uint32_t *hits, uint64_t hits_cap);
/* Capture one mb_plan_run with these inputs into a CUDA graph kept by the plan; mb_plan_replay
 * launches that graph on `stream` (the inputs are read again from the same device buffers). */
int mb_plan_capture(mb_plan *plan, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                    const uint8_t *mate);
int mb_plan_replay(mb_plan *plan, void *stream);
int mb_autotune(const mb_index *idx, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                const mb_opts *opts, void *stream, mb_opts *best, double *best_ms);
int mb_autotune_points(const mb_index *idx, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                       const mb_opts *opts, void *stream, mb_opts *best, double *best_ms, mb_opts *points,
                       double *points_ms, uint32_t cap, uint32_t *n_points);

/* ---------------------------------------------------------------------------------------
 * Served form: continuous batching of seeding requests on one GPU.
 * mb_serve_create starts a worker thread and a helper thread and allocates a 1 GiB pinned host
 * ring in which submitted bases wait.  Device work runs in execution slots (a stream and a seeding
 * plan for up to 65,536 reads / 64M bases / 2M SMEMs / 32M hits each, about 0.8 GB of device
 * memory; at most 32 slots).  Slots are admitted by free device memory: a slot is created only when requests wait
 * and every slot is busy, and only while cudaMemGetInfo's free bytes minus a reserve left to other
 * users (2% of the device, at least 1 GiB) hold one more slot and the slots stay within
 * hbm_budget bytes (0 = no budget; one slot is always allowed by the budget); otherwise requests
 * wait until a slot frees.  Idle slots are released while free memory is below the reserve.
 * Whenever a slot is free, the oldest waiting request and the later ones of its kind that still
 * fit the slot's limits are merged into one launch group, so requests arriving while others are
 * on the GPU are admitted as soon as a slot frees, and groups run concurrently on their own
 * streams.  The kinds: requests with a read of 1,000 bases or more, and the others; a group takes
 * as long as its longest read, so requests of short reads are never grouped with long reads, and
 * groups of long reads hold at most half of the slots at a time.  Each slot runs its plan as one
 * CUDA graph captured for the slot's 65,536 reads (a smaller group pads its offsets with empty
 * reads), so a group costs one graph launch on the worker thread.  A group whose records or hits
 * exceed its plan is seeded again request by request on the helper thread (allocating entry
 * points), so the worker keeps serving.  Each request's results are exactly those of
 * mb_seed_batch + mb_locate on that request alone (read numbers and hit offsets relative to it).
 *   mb_serve_submit  copies the request's bases into the pinned ring on the calling thread and
 *                    returns a ticket at once.  MB_ERR_ARG if the request alone exceeds a slot's
 *                    limits; MB_ERR_BUSY if the ring has no room for it now (too many bases are
 *                    outstanding: collect results and submit again).
 *   mb_serve_poll    *done = 1 when the ticket's results are ready.
 *   mb_serve_wait    waits up to timeout_ms (0 = no limit; MB_ERR_TIMEOUT after it) and returns
 *                    server-owned host arrays valid until mb_serve_release(ticket), plus the
 *                    request's latency from submit to results ready, in ms.
 *   mb_serve_destroy finishes every request already submitted, then stops and frees the server.
 * Every call on a server that was destroyed (or never created) returns MB_ERR_ARG without
 * touching it.
 */
int mb_serve_create(const mb_index *idx, const mb_opts *opts, uint64_t hbm_budget, mb_server **out);
int mb_serve_submit(mb_server *srv, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                    uint64_t *ticket);
int mb_serve_poll(mb_server *srv, uint64_t ticket, int *done);
int mb_serve_wait(mb_server *srv, uint64_t ticket, uint32_t timeout_ms, const mb_smem **smem,
                  uint64_t *n_smem, const uint32_t **hits, uint64_t *n_hits, double *latency_ms);
int mb_serve_release(mb_server *srv, uint64_t ticket);
int mb_serve_destroy(mb_server *srv);
/* slots = execution slots now; groups = launch groups run; merged = requests that shared a group
 * with another request (the continuous-batching count). */
int mb_serve_stats(mb_server *srv, uint32_t *slots, uint64_t *groups, uint64_t *merged);
/* Up to `count` counters, in this order: slots now, groups, merged, slots created, slots released,
 * slot allocations that failed, groups that outgrew their plan, submits refused with MB_ERR_BUSY,
 * ms that waiting requests spent with every slot busy and no memory for another, device bytes of
 * one slot, the free-memory reserve in bytes, groups of requests with long reads, ms the worker
 * thread spent launching groups and handing out results (13 exist). */
int mb_serve_counters(mb_server *srv, uint64_t *out, uint32_t count);
/* Fault injection for tests of admission (no counterpart in the paper): from now on admission sees
 * free_bytes of free device memory instead of cudaMemGetInfo's value (free_bytes < 0 restores the
 * real query), and the next fail_slots slot creations fail as an allocation failure would. */
int mb_serve_inject(mb_server *srv, int64_t free_bytes, uint32_t fail_slots);

/* Section 2.9 strand rule on the 3-base index: keep[h] = 1 if hit h of an SMEM of read `mate`
 * 1 lies wholly inside the forward C-to-T or the reverse G-to-A copy of the reference (read 2:
 * forward G-to-A or reverse C-to-T), else 0.  All pointers host or device. */
int mb_bs_filter(const mb_index *idx, const mb_smem *smem, uint64_t n_smem, const uint8_t *mate,
                 const uint32_t *hits, uint64_t n_hits, void *stream, uint8_t *keep);

/* One piece of a split bisulfite seed (24 bytes): read[qbeg, qend) matches the text at pos; hit
 * is the index of the seed's hit in mb_locate's output. */
typedef struct {
    uint64_t hit;
    uint32_t read, qbeg, qend, pos;
} mb_piece;

/* ---------------------------------------------------------------------------------------
 * mb_bs_split — Section 2.9: a seed found on the 3-base index may pair a read C with a
 * reference T (read 1, C->T converted) or a read G with a reference A (read 2, G->A); such a
 * T-to-C mismatch is not a bisulfite conversion.  For every hit h with keep[h] != 0 (keep may
 * be NULL: every hit), the original read bases under the seed are compared with the original
 * reference bases under the hit: for a hit in copy g = pos / |R| of the text
 * CT(R) GA(R) rc(GA(R)) rc(CT(R)) $ at offset q = pos - g|R|, copies 0 and 1 give R[q + t],
 * copies 2 and 3 the complement of R[|R| - 1 - (q + t)].  The seed is cut at every read C over
 * a reference T (reads with mate 1) or read G over a reference A (mate 2); the cut base belongs
 * to no piece; reads with mate 0 are not cut.  Pieces of at least opts->min_len (default 19)
 * bases are written in hit order, then qbeg order; pos is the piece's text position.  A hit that
 * does not lie inside one copy gives no piece.
 *   ref          host or device, the |R| original reference codes (0..3; > 3 = N, never cuts)
 *                the MB_BS3 index was built from.
 *   seq, off, mate, smem, hits: the original (unconverted) reads and the outputs of
 *                mb_seed_batch / mb_locate; keep: the output of mb_bs_filter or NULL.
 *   out          host or device, room for `cap` pieces; *n_out receives the count (if it
 *                exceeds cap: MB_ERR_CAPACITY, nothing written).
 * Errors: MB_ERR_ARG (also for an index built without MB_BS3), MB_ERR_CAPACITY, MB_ERR_NOMEM,
 * MB_ERR_CUDA.
 */
int mb_bs_split(const mb_index *idx, const uint8_t *ref, const uint8_t *seq, const uint64_t *off,
                uint32_t n_reads, const uint8_t *mate, const mb_smem *smem, uint64_t n_smem,
                const uint32_t *hits, const uint8_t *keep, uint64_t n_hits, const mb_opts *opts,
                void *stream, mb_piece *out, uint64_t cap, uint64_t *n_out);

/* ---------------------------------------------------------------------------------------
 * mb_rescue_prefilter — the mate-rescue prefilter of Section 2.7: for each pair p of a read
 * P = reads[read_off[p], read_off[p+1]) and a reference window R = wins[win_off[p],
 * win_off[p+1]), best[p] = max over t of M_t = #{(i, j) : P[i, i+q) = R[j, j+q), j - i = t}
 * (0 when no q-mer matches), over every q-mer start i of P and j of R.  A q-mer holding an N
 * (code > 3) matches nothing.  The paper starts a Smith-Waterman alignment only when
 * best >= 10 with q = 7.  Independent of any index.
 *   reads, wins, read_off, win_off: host or device; offsets non-decreasing.
 *   q        1..15 (0 = 7).
 *   best     host or device, n_pairs u32.
 * The longest read plus the longest window, 4 bytes per base, must fit one block's shared
 * memory (e.g. reads of 1 kb with windows of 50 kb).
 * Errors: MB_ERR_ARG, MB_ERR_NOMEM, MB_ERR_CUDA.
 */
int mb_rescue_prefilter(const uint8_t *reads, const uint64_t *read_off, const uint8_t *wins,
                        const uint64_t *win_off, uint32_t n_pairs, uint32_t q, void *stream,
                        uint32_t *best);

/* Map a text position to the reference: strand 0 = forward, 1 = reverse complement;
 * rpos = the start on the forward strand of the match of length len. */
int mb_hit_to_ref(const mb_index *idx, uint64_t pos, uint64_t len, int *strand, uint64_t *rpos);

const char *mb_strerror(int code);

/* Set the L2 fetch granularity of the calling process's CUDA context on the current device
 * (cudaLimitMaxL2FetchGranularity; 32, 64 or 128 bytes; 0 leaves it unchanged) and return the
 * value in force in *now.  Every block access of the seeding kernels is a random 32-byte read;
 * with a larger granularity the L2 fetches the rest of the line from DRAM for nothing.  The
 * limit belongs to this process's context only (other processes and later users of the GPU are
 * not affected) but it applies to every kernel of this process.  No counterpart in the paper. */
int mb_set_l2_fetch_granularity(int bytes, int *now);
/* The device allocation holding device pointer p: [*base, *base + *size), as the driver reports it.
 * Every entry point checks its device buffers this way before a kernel touches them (a span that
 * passes the end of its allocation gives MB_ERR_ARG).  MB_ERR_ARG for host or null pointers,
 * MB_ERR_CUDA when the driver cannot tell (then those checks are skipped).  No counterpart in the
 * paper. */
int mb_device_extent(const void *p, uint64_t *base, uint64_t *size);
/* L2 persistence for the k-mer ds-interval table (Section 2.5 keeps it in a CPU cache): sets an
 * access-policy window on `stream` over the first min(max_bytes, table bytes, the device's window
 * and persisting-L2 limits) bytes of the table, hits persisting, and sets this context's
 * persisting-L2 limit to that size (*window receives it).  Kernels later launched on `stream`
 * keep those table lines in L2.  max_bytes = 0 removes the window and resets persisting lines.
 * Like mb_set_l2_fetch_granularity this changes only the calling process's context.  No
 * counterpart in the paper. */
int mb_index_l2_persist(const mb_index *idx, void *stream, uint64_t max_bytes, uint64_t *window);
/* Detail of the last error of this library (host-side message), for diagnostics. */
const char *mb_last_error(void);

/* ---------------------------------------------------------------------------------------
 * Measurement hooks (no effect on results).
 * mb_profile_enable(1): CUDA events are recorded on the launching stream around the SMEM
 * kernel ("smem") and the locate kernel ("locate"); mb_profile_get returns the summed
 * device time in ms and the number of timed launches since the last reset.
 * mb_launch_count: number of kernels this library has launched since it was loaded.
 * mb_work_counters: work done by calls made with MB_COUNT in opts, summed since the last
 * reset: extension steps of Algorithm 3, distinct occurrence blocks they read, k-mer table
 * lookups, LF steps of Algorithm 2 and sampled-SA reads.
 * mb_work_counters_all: the same five followed by the work of extending unique matches by text
 * comparison (LF steps of its walks, SA / ISA sample reads, text loads of 8 bytes), then of the
 * locate walks that join (walks that stopped at a walked row of an earlier pass, each reading that
 * row's rank and position; calls whose walked rows were not sorted and distinct, so that no walk
 * joined), `count` values at most (10 exist).  The LF steps and sampled-S reads are those of the
 * walks run: exactly Algorithm 2's over the distinct rows, or fewer with MB_LOCATE_JOIN.
 */
void mb_profile_enable(int on);
int mb_profile_get(const char *kernel, double *ms, uint64_t *launches);
void mb_profile_reset(void);
uint64_t mb_launch_count(void);
void mb_work_counters(uint64_t *ext_steps, uint64_t *ext_blocks, uint64_t *kmer_lookups,
                      uint64_t *lf_steps, uint64_t *sa_reads);
void mb_work_counters_all(uint64_t *out, uint32_t count);

#ifdef __cplusplus
}
#endif
#endif
