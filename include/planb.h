/*
 * planb.h — C ABI of libplanb.so: batched IPv6 longest-prefix-match (LPM) on a GB300 (sm_103a) GPU,
 * by the PlanB method (arXiv 2604.14650): prefixes are turned into sorted elementary intervals
 * (Section 3.1) and stored as a flat-array linearized B+-tree (Section 3.2) that a CUDA kernel
 * descends once per 128-bit destination address (Algorithm 1) to that interval's next hop.
 *
 * Conventions shared by every call
 *   - Addresses and prefixes are 128-bit numbers held as two uint64_t halves: `hi` is the first
 *     8 bytes of the address in network order read as a big-endian integer, `lo` the last 8
 *     (Section 3.1's example: 2001:db8:: is hi = 0x20010db800000000, lo = 0).
 *   - A prefix is (hi, lo, len) with len in 0..128; host bits beyond len are ignored (masked).
 *     When the same (prefix, len) is given more than once, the last one wins.
 *   - An address that no prefix covers gets the ::/0 next hop when the table has one, else 0
 *     (Section 3.1: uncovered intervals take the default route).
 *   - Return value: 0 (PLANB_OK) on success, a negative PLANB_E* code on failure; planb_strerror()
 *     names it. A failed call changes nothing the caller can observe, except where stated.
 *   - `stream` is a cudaStream_t (0 = the legacy default stream). Calls that take one are
 *     asynchronous with respect to the host: results are ready when the stream has completed.
 *   - Host pointers are read during the call only; the library keeps no reference to them.
 *     Device pointers (the d_ arguments) are caller-owned device memory on the fib's device.
 */
#ifndef PLANB_H
#define PLANB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *planb_stream_t; /* same type as cudaStream_t */

/* ----------------------------------------------------------------------------- status codes */
#define PLANB_OK 0
#define PLANB_EINVAL (-1)   /* null pointer, len > 128, size too large, bad option            */
#define PLANB_ENOMEM (-2)   /* host or device allocation failed                               */
#define PLANB_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed                     */
#define PLANB_EDEVICE (-4)  /* a kernel reported an error through the fib's device status word */
#define PLANB_ENODEV (-5)   /* no CUDA device, or the device is not sm_103                      */
#define PLANB_ETIMEOUT (-6) /* a bounded device-side wait ran out                               */

/* ----------------------------------------------------------------------------- node formats */
/* F8x128: 8 full 128-bit keys per 128-byte node, 9-ary (the paper's k = 8, b = 9 of Section 3.2,
 * with 128-bit keys instead of the 64-bit key halves the paper uses). */
#define PLANB_FMT_F8X128 0
/* F16HI: 16 key high halves per 128-byte node, 17-ary (Section 3.2: 128-byte lines give 16-key,
 * 17-ary nodes); a parallel array holds the low halves. Lookups count keys by their high halves
 * alone. The next hops are 32-bit words whose bit 16 marks an interval whose key (its inclusive
 * end) has a low half other than all-ones (a /65../128 boundary): only at such a count can a key
 * that shares the address's high half still be below the address, and only there are the low
 * halves (the key's and the address's) read. */
#define PLANB_FMT_F16HI 1
/* F8V7: internal nodes as F8X128; each 128-byte leaf line holds 7 keys and, in its last
 * 16 bytes, the 7 next hops of those keys. The paper keeps values in a separate array (Section 3.2,
 * "Separation of Keys and Values") and fetches one after the descent; packing them into the leaf
 * line removes that dependent memory access. The last interval gets an explicit all-ones key, so the
 * count at a leaf is always 0..6 and names a slot of that same line. Hybrid kernel only. */
#define PLANB_FMT_F8V7 2

/* ----------------------------------------------------------------------------- lookup kernels */
#define PLANB_KERNEL_AUTO 0   /* hybrid                                                            */
/* coop: every level by 8-lane (16-lane for F16HI) groups, one coalesced 128-byte node line per
 * level (Listing 1's node search as a warp ballot + popcount), top levels staged in shared memory */
#define PLANB_KERNEL_COOP 1
/* hybrid (F8X128, F8V7, F16HI): the top S levels are replaced by a per-thread lower bound over the
 * level-S subtree maxima held in shared memory (the same count, so the same node), started in the
 * address's bucket of a radix directory; the remaining levels are descended cooperatively from L2
 * with several addresses per lane group in flight. With F16HI (16 keys per leaf) the index over
 * the leaves of a 200k-prefix table fits one CTA's shared memory, leaving the leaf line alone in
 * L2; such tables run one 1024-thread CTA per SM (an index too large for the multi-table kernel's
 * shared memory makes a multi-table group give that table a launch of its own). */
#define PLANB_KERNEL_HYBRID 2
/* flat (F8X128 only): per-thread binary search over the sorted interval keys in global memory;
 * the GPU analogue of the paper's ablation baseline (Section 4.5, std::lower_bound) */
#define PLANB_KERNEL_FLAT 3
/* learned (F8X128 or F8V7): the hybrid kernel whose shared-memory search starts from a learned
 * position model — a two-layer recursive model index (a 16-unit FP32 MLP root trained on the GPU
 * at build time, linear leaves) that predicts each address's interval rank with a recorded per-leaf
 * error bound; a bounded search inside that window fixes the rank exactly, and leaves whose bound
 * exceeds 64 ranks (or addresses the window does not bracket) take the plain tree path. The paper
 * has no learned component; this follows the learned-index idea on top of its tree. */
#define PLANB_KERNEL_LEARNED 4

/* Builders (planb_opts.builder). Both give the same table, word for word.
 * host: the prefix sort and Algorithm 2's stack sweep run on the host (Section 3.6), then the
 *   layout is filled on the host and uploaded.
 * device: every build step runs on the GPU: radix sorts of the prefixes and of the range-end
 *   events, the stack sweep replaced by a bracket-matching scan (nesting depth by a prefix sum,
 *   then for every event the latest start at the same depth), and the node arrays, index and
 *   next hops written in place by closed-form kernels. Device scratch is about 120 bytes per
 *   prefix during the build. Rebuilds by planb_update use the same builder. */
#define PLANB_BUILDER_HOST 0
#define PLANB_BUILDER_DEVICE 1

typedef struct planb_fib planb_fib; /* opaque; owns all host and device memory of one table */

typedef struct {
    uint32_t struct_size;   /* sizeof(planb_opts); lets the library accept older callers        */
    int32_t format;         /* PLANB_FMT_*; default PLANB_FMT_F8X128 (every kernel takes it);
                               PLANB_FMT_F16HI with the hybrid kernel is the fastest lookup     */
    int32_t merge_equal_nh; /* 1: merge neighbouring intervals with equal next hops (Section 3
                               intro allows compressing routes that share a next hop); results
                               are unchanged. Default 0.                                        */
    int32_t smem_levels;    /* tree levels resolved in shared memory per CTA (coop: levels staged;
                               hybrid: levels replaced by the index); -1 = automatic            */
    int32_t device;         /* CUDA device ordinal; -1 = the current device                      */
    int32_t block_threads;  /* threads per CTA of the lookup kernel; 0 = automatic               */
    int32_t ctas_per_sm;    /* persistent CTAs per SM; 0 = as many as fit                        */
    int32_t kernel;         /* PLANB_KERNEL_*; default PLANB_KERNEL_AUTO                          */
    int32_t model_leaves;   /* learned: leaf models L; 0 = automatic                              */
    int32_t model_iters;    /* learned: Adam steps of the root's training; -1 = default (2000)    */
    int32_t builder;        /* PLANB_BUILDER_*: where the build steps run; default host          */
    int32_t reserved[4];    /* zero                                                              */
} planb_opts;

/* Fills *o with the defaults. */
void planb_opts_default(planb_opts *o);

typedef struct {
    uint64_t n_input;          /* prefixes given to the last (re)build                           */
    uint64_t n_prefixes;       /* distinct canonical prefixes in the table                       */
    uint64_t n_intervals;      /* elementary intervals m (Section 3.1: at most 2N + 1)            */
    uint32_t depth;            /* levels D including the leaf level (Algorithm 1 visits D nodes)  */
    uint32_t keys_per_node;    /* k                                                              */
    uint32_t fanout;           /* b = k + 1                                                      */
    uint32_t smem_levels;      /* levels staged in shared memory by the lookup kernel            */
    uint32_t format;           /* PLANB_FMT_*                                                    */
    uint32_t device;           /* device ordinal                                                 */
    uint64_t internal_nodes;   /* nodes of the internal levels (complete levels, Section 3.2)     */
    uint64_t leaf_nodes;       /* leaf nodes allocated (trailing all-padding leaves are not)      */
    uint64_t node_bytes;       /* bytes of the node array(s) on the device                       */
    uint64_t value_bytes;      /* bytes of the next-hop array on the device                      */
    uint64_t version;          /* table generation: 1 after build, +1 per applied update         */
    uint64_t withdraw_absent;  /* withdraws of prefixes that were not in the table (no-ops)       */
    double build_ms;           /* wall time of the last build: host builder, canonicalise ..
                                  layout on the host; device builder, every step incl. the fill */
    double upload_ms;          /* host builder: time to allocate and upload the last table;
                                  device builder: 0 (the fill is part of build_ms)               */
    uint32_t kernel;           /* PLANB_KERNEL_* in use (never AUTO)                             */
    uint32_t threads;          /* threads per CTA of the lookup kernel                           */
    uint32_t ctas;             /* persistent grid size (CTAs)                                    */
    uint32_t smem_bytes;       /* dynamic shared memory per CTA                                  */
    uint32_t model_leaves;     /* learned: leaf models (0 for the other kernels)                 */
    uint32_t model_iters;      /* learned: Adam steps run                                        */
    uint32_t model_max_err;    /* learned: largest per-leaf bound, in ranks                      */
    uint32_t builder;          /* PLANB_BUILDER_* that made the current table                    */
    double model_loss0;        /* learned: root's mean squared CDF error before training         */
    double model_loss;         /* learned: ... and after                                         */
    double model_covered;      /* learned: share of keys in leaves within the window limit       */
    double model_mean_err;     /* learned: mean bound over those keys                            */
    double model_train_ms;     /* learned: training time (GPU)                                   */
} planb_stats_t;

/*
 * planb_build — builds a table from n prefixes and uploads it to the device.
 *   prefix_hi, prefix_lo, len, nexthop: host arrays of n entries (n may be 0: every address then
 *     gets next hop 0). opts may be NULL for the defaults.
 *   *out receives the new table; the caller frees it with planb_destroy.
 * Steps (Section 3.1 "Range Conversion" and "Interval Partitioning"; Section 3.6, Algorithm 2):
 * each prefix P/L becomes the range [P, P + 2^(128-L)), the range ends become sorted boundaries,
 * a sweep assigns each elementary interval the next hop of its longest covering prefix, and the
 * interval bounds are laid out as a linearized B+-tree (Section 3.2).
 * Errors: PLANB_EINVAL (null pointer with n > 0, len > 128, bad option), PLANB_ENOMEM,
 *   PLANB_ENODEV, PLANB_ECUDA.
 */
int planb_build(const uint64_t *prefix_hi, const uint64_t *prefix_lo, const uint8_t *len,
                const uint16_t *nexthop, size_t n, const planb_opts *opts, planb_fib **out);

/*
 * planb_lookup — next hop of n addresses (Algorithm 1, Section 3.2; value fetch of "Separation of
 * Keys and Values", Section 3.2).
 *   d_addr_hi, d_addr_lo: device arrays of n uint64_t (8-byte aligned); d_out: device array of n
 *   uint16_t (2-byte aligned). n = 0 is a no-op. Enqueued on `stream`; returns before it runs.
 *   It uses the table that is current when the call is made (see planb_update).
 * Errors: PLANB_EINVAL (null pointer with n > 0, misaligned pointer), PLANB_ECUDA (launch failed).
 */
int planb_lookup(const planb_fib *fib, const uint64_t *d_addr_hi, const uint64_t *d_addr_lo,
                 size_t n, uint16_t *d_out, planb_stream_t stream);

/*
 * planb_lookup_host — the same lookup for addresses and results in HOST memory. When all three
 * buffers are page-locked and device-addressable, the lookup kernel reads the addresses and writes
 * the next hops over the host link itself, as planb_lookup_mapped does (an address's low half is
 * read only on a tie of high halves). Otherwise the library copies the addresses to the device in
 * chunks, runs the lookup kernel on each chunk and copies the next hops back, overlapping the
 * copies of one chunk with the lookup of another on its own streams. Either way it returns when
 * every result is in `out` (synchronous).
 *   addr_hi, addr_lo: host arrays of n uint64_t; out: host array of n uint16_t.
 *   The device staging buffers are owned by the fib and reused by later calls.
 * Errors: PLANB_EINVAL, PLANB_ENOMEM, PLANB_ECUDA.
 */
int planb_lookup_host(planb_fib *fib, const uint64_t *addr_hi, const uint64_t *addr_lo, size_t n,
                      uint16_t *out);

typedef struct {
    uint64_t hi, lo;
    uint8_t len;
    uint16_t nexthop;
} planb_route; /* an insert, or a modify when (prefix, len) is already present (Section 3.6) */

typedef struct {
    uint64_t hi, lo;
    uint8_t len;
} planb_prefix; /* a withdraw; a prefix that is not present (including one already withdrawn
                   earlier in the same batch) is a counted no-op */

/*
 * planb_lookup_mapped — planb_lookup on page-locked host buffers, read and written by the lookup
 * kernel itself over the host link (on a Grace-Blackwell node, NVLink-C2C) instead of being copied:
 * the address stream goes straight from host memory into the descent and the next hops straight
 * back. addr_hi, addr_lo, out: host arrays of n entries in page-locked memory the device can address
 * (cudaHostAlloc, or cudaHostRegister with the mapped flag; a PyTorch pinned tensor); asynchronous
 * on `stream` like planb_lookup. The paper has no counterpart (its lookups run where the packets
 * are). Errors: PLANB_EINVAL (null, misaligned, or a buffer that is not such memory: nothing is
 * launched), PLANB_ECUDA.
 */
int planb_lookup_mapped(const planb_fib *fib, const uint64_t *addr_hi, const uint64_t *addr_lo,
                        size_t n, uint16_t *out, planb_stream_t stream);

/*
 * planb_update — applies a batch of route changes by rebuild-and-swap (Section 3.6, "Dynamic FIB
 * Update"): the changes are merged into the table's canonical prefix list (withdraws first, then
 * inserts, each batch in order), a complete new table is built and uploaded, and the fib is
 * switched to it with one pointer swap. Lookups enqueued before the call keep using the old
 * table; lookups enqueued after it return use the new one. The old table is freed only after the
 * work already enqueued on every stream this fib's lookups have used (and on `stream`) is done.
 *   inserts: host array of n_ins routes; withdraws: host array of n_wd prefixes (either may be
 *   NULL when its count is 0).
 * On any failure the previous table stays current and unchanged.
 * Errors: PLANB_EINVAL (len > 128, null pointer with a count > 0), PLANB_ENOMEM, PLANB_ECUDA.
 */
int planb_update(planb_fib *fib, const planb_route *inserts, size_t n_ins,
                 const planb_prefix *withdraws, size_t n_wd, planb_stream_t stream);

/*
 * planb_forget_stream — the fib fences table retirement (planb_update) on every stream its
 * lookups have used, so such a stream must stay valid while it is remembered. Before destroying a
 * stream that was used with this fib (planb_lookup, planb_update, or a planb_multi_lookup over
 * it), call this: it waits for the stream's queued work and removes the stream from the set. The
 * paper has no counterpart (it frees the old table after its readers finish, Section 3.6).
 * Errors: PLANB_EINVAL (null fib), PLANB_ECUDA.
 */
int planb_forget_stream(planb_fib *fib, planb_stream_t stream);

/* planb_stats — copies the table's statistics into *out. Errors: PLANB_EINVAL. */
int planb_stats(const planb_fib *fib, planb_stats_t *out);

/*
 * planb_device_status — waits for the device, then reads and clears the fib's device status word,
 * which kernels set when a bounds check fails (builds with PLANB_BOUNDS_CHECK) or a bounded wait
 * runs out. Returns PLANB_OK, PLANB_EDEVICE or PLANB_ETIMEOUT; *detail (nullable) receives the
 * raw word.
 */
int planb_device_status(planb_fib *fib, uint32_t *detail);

/* planb_destroy — waits for the fib's outstanding work and frees it. NULL is a no-op. */
void planb_destroy(planb_fib *fib);

/* planb_strerror — a static string naming a PLANB_* code. */
const char *planb_strerror(int code);

/* planb_last_error — where the last failing call on this thread failed, with the CUDA error text
 * when there was one ("" if none recorded). The string belongs to the library and stays valid until
 * the next failing call on the same thread. */
const char *planb_last_error(void);

/* ------------------------------------------------------------------------ multi-table lookups */

typedef struct planb_multi planb_multi; /* several tables (VRFs) served by one captured graph */

/*
 * planb_multi_create — groups n_tables built tables (all on one device) for lookups whose
 * addresses each carry a u8 table id. The paper serves one table; many tables per box are the
 * same lookup applied per table. fibs: n_tables table handles (1..255), not owned: they must
 * outlive the group; updates to them are picked up by later lookups. max_batch: most addresses per
 * planb_multi_lookup call (< 2^32); the group owns about max_batch x 16.2 bytes of device scratch
 * (plus about 3 bytes per address per 1,000 tables).
 * Tables built with PLANB_KERNEL_LEARNED cannot join a group. flags: 0, or an OR of the
 * PLANB_MULTI_* flags below. Errors: PLANB_EINVAL, PLANB_ENOMEM, PLANB_ECUDA.
 */
#define PLANB_MULTI_NO_GRAPH 1u  /* flag: launch the pipeline directly instead of a captured graph */
#define PLANB_MULTI_PER_TABLE 2u /* flag: one lookup launch per table even where every table could
                                    share the single persistent launch (for comparison)          */
#define PLANB_MULTI_BUCKETED 4u  /* flag: group the batch by table even where every table could
                                    take the direct launch (for comparison)                      */
#define PLANB_MULTI_DIRECT 8u    /* flag: the direct launch at every batch size where the tables
                                    allow it (for comparison)                                    */
int planb_multi_create(planb_fib *const *fibs, uint32_t n_tables, size_t max_batch,
                       uint32_t flags, planb_multi **out);

/*
 * planb_multi_lookup — next hop of n addresses, address i looked up in table d_table[i]
 * (ids >= n_tables give 0). d_addr_hi, d_addr_lo: device u64 arrays; d_table: device u8 array;
 * d_out: device u16 array; all of n entries. Three forms (planb_multi_mode):
 *  - direct: when every table is an F16HI table of the hybrid kernel (of fewer than 2^24 nodes,
 *    about 268 million keys), one persistent launch looks up the batch in input order, each
 *    address in its own table through that table's in-place index, and writes each result at its
 *    input position. It reads every table's lines at once, so it is taken while those fit in L2
 *    (at most 32 MB of leaf high halves, next-hop words and index) or the batch has at most 2^24
 *    addresses (max_n for planb_multi_lookup_devn), and at every size with PLANB_MULTI_DIRECT;
 *  - bucketed: else, the batch is grouped by table (a counting sort on the device). When every
 *    table uses the hybrid kernel (any format), one persistent launch looks up all groups: the
 *    CTAs claim pieces of the grouped batch in order and stage the index of each table they meet;
 *    results are gathered back into the input order;
 *  - per-table: else, each table's group gets its own launch.
 * The whole pipeline is captured once as a CUDA graph and replayed while the buffers and n stay
 * the same. In the single-launch forms, a table swapped by planb_update reaches the replays
 * through its record (copied in stream order). New buffers, a change of the launch's shape, or a
 * swap under per-table launches cause one new capture. Enqueued on
 * `stream`; calls on one group are serialised on the host, and since the group's device scratch
 * is reused by every call, all calls on one group must use the same stream.
 * Errors: PLANB_EINVAL (null pointer, misalignment, n > max_batch), PLANB_ECUDA.
 */
int planb_multi_lookup(planb_multi *m, const uint64_t *d_addr_hi, const uint64_t *d_addr_lo,
                       const uint8_t *d_table, size_t n, uint16_t *d_out, planb_stream_t stream);

/*
 * planb_multi_lookup_devn — planb_multi_lookup with the batch size read from device memory
 * (*d_n, a uint64_t written before the work runs, at most max_n <= max_batch): the captured graph
 * depends on the buffers and max_n only, so batches of any size replay it without a new capture
 * (a serving loop's slots do this). Errors as planb_multi_lookup.
 */
int planb_multi_lookup_devn(planb_multi *m, const uint64_t *d_addr_hi, const uint64_t *d_addr_lo,
                            const uint8_t *d_table, const uint64_t *d_n, size_t max_n,
                            uint16_t *d_out, planb_stream_t stream);

/* planb_multi_persistent — 1 when the group's lookups run as a single persistent launch (the
 * direct or the bucketed form of planb_multi_lookup), 0 when each table gets its own launch.
 * Decided at the first lookup and again whenever a table is swapped; 0 before the first lookup.
 * Errors: PLANB_EINVAL. */
int planb_multi_persistent(const planb_multi *m);

/* planb_multi_mode — the form of the group's last lookup: PLANB_MULTI_MODE_DIRECT,
 * PLANB_MULTI_MODE_BUCKETED (grouped by table, one persistent launch) or
 * PLANB_MULTI_MODE_PER_TABLE (also before the first lookup). Errors: PLANB_EINVAL. */
#define PLANB_MULTI_MODE_PER_TABLE 0
#define PLANB_MULTI_MODE_BUCKETED 1
#define PLANB_MULTI_MODE_DIRECT 2
int planb_multi_mode(const planb_multi *m);

/* planb_multi_captures — how many times the group has captured its graph (the first lookup,
 * then once per table swap or buffer change seen by a lookup); 0 for NULL. */
uint64_t planb_multi_captures(const planb_multi *m);

/* planb_multi_destroy — waits for the device and frees the group (not its tables). */
void planb_multi_destroy(planb_multi *m);

/* ------------------------------------------------------------------------------ serving loop */

typedef struct planb_server planb_server;

typedef struct {
    uint32_t struct_size;      /* sizeof(planb_server_opts)                                      */
    uint32_t slots;            /* batches in flight at once, each on its own stream; default 4    */
    uint32_t max_batch;        /* addresses per device batch; default 262,144                     */
    uint32_t max_request;      /* addresses per request (<= max_batch); default 65,536            */
    uint64_t mem_budget;       /* device bytes the admitted tables may hold; 0 = no limit         */
    uint32_t update_period_us; /* how often queued route changes are applied; default 10,000      */
    int32_t device;            /* CUDA device; -1 = current                                       */
    uint32_t multi_flags;      /* flags of the slots' table groups (PLANB_MULTI_*); default 0     */
    uint32_t reserved[5];
} planb_server_opts;

typedef struct {
    uint64_t requests, lookups, batches;  /* completed since start (or the last reset)          */
    uint64_t updates, update_batches;     /* route changes applied, rebuilds run                 */
    uint64_t tables, table_bytes, queued; /* admitted tables, their device bytes, queue depth    */
    double p50_us, p99_us, max_us;        /* request latency, submit to results in place         */
    double mean_batch;                    /* addresses per device batch                          */
    double rebuild_ms_mean;               /* mean time of one table's rebuild-and-swap           */
    int32_t last_error;                   /* last failure code inside the engine (0 = none)      */
    int32_t reserved;
    double batch_p50_us, batch_p99_us, batch_max_us; /* device batches, launch to results seen  */
    uint64_t recaptures;                  /* slot graph captures after a table swap              */
} planb_server_stats_t;

void planb_server_opts_default(planb_server_opts *o);

/*
 * planb_server_create — a serving engine: continuous batching of lookup requests over a set of
 * tables (the paper's data plane batches NIC bursts, Section 3.4, and applies route changes by
 * rebuild-and-swap, Section 3.6). Requests queue up; a dispatcher thread packs whatever is queued
 * into the next free slot (pinned staging + device buffers of max_batch addresses on its own
 * stream), so requests arriving while others run join the next batch, and the slots' copies and
 * lookups overlap on the device. A slot runs one multi-table pipeline (planb_multi_lookup_devn) per
 * batch. An updater thread applies queued route changes every update period; batches formed after
 * a table's swap see the new table. Errors: PLANB_EINVAL, PLANB_ENOMEM, PLANB_ENODEV, PLANB_ECUDA.
 */
int planb_server_create(const planb_server_opts *opts, planb_server **out);

/*
 * planb_server_add_table — admits a built table (same device) if the tables' device bytes stay
 * within mem_budget; *table_id receives its id (0, 1, ...). Not owned: it must outlive the server.
 * Errors: PLANB_EINVAL (255 tables already, other device), PLANB_ENOMEM (over the budget: not
 * admitted).
 */
int planb_server_add_table(planb_server *s, planb_fib *fib, uint32_t *table_id);

/*
 * planb_server_submit — queues a request: the next hops of n (1..max_request) addresses in table
 * table_id. addr_hi, addr_lo, out: host arrays that must stay valid until planb_server_wait reports
 * the request done. Returns at once; *ticket identifies the request.
 * Errors: PLANB_EINVAL, PLANB_ENOMEM.
 */
int planb_server_submit(planb_server *s, uint32_t table_id, const uint64_t *addr_hi,
                        const uint64_t *addr_lo, size_t n, uint16_t *out, uint64_t *ticket);

/*
 * planb_server_wait — waits up to timeout_us for a request; returns PLANB_OK when its results are
 * in place (the ticket is then released), PLANB_ETIMEOUT if still running, else the failure code.
 */
int planb_server_wait(planb_server *s, uint64_t ticket, uint32_t timeout_us);

/*
 * planb_server_update — queues route changes for a table (applied by the updater thread at the
 * next update period, all changes queued for the table in one rebuild). Errors: PLANB_EINVAL.
 */
int planb_server_update(planb_server *s, uint32_t table_id, const planb_route *inserts,
                        size_t n_ins, const planb_prefix *withdraws, size_t n_wd);

/* planb_server_stats — counters and latency percentiles (over the last 2^20 requests). */
int planb_server_stats(planb_server *s, planb_server_stats_t *out);

/* planb_server_error_detail — copies (NUL-terminated, truncated to cap) where and why the engine
 * last failed: the failing step and the CUDA error, or "" when nothing failed. Errors:
 * PLANB_EINVAL. */
int planb_server_error_detail(planb_server *s, char *buf, size_t cap);

/* planb_server_reset_stats — zeroes the counters and the latency record. */
void planb_server_reset_stats(planb_server *s);

/* planb_server_destroy — stops the threads, finishes the batches in flight and frees the engine
 * (not its tables); requests still queued fail with PLANB_EINVAL. */
void planb_server_destroy(planb_server *s);

/* ------------------------------------------------------ learned-model kernels (for checking) */

/*
 * planb_mlp_grad — the training kernels' full-batch gradient: for the root MLP
 * y(u) = b2 + sum_h w2[h] min(max(w1[h] u + b1[h], 0), cap[h]) (16 saturating ReLU units) and the
 * loss L = (1/n) sum_i (y(u_i) - t_i)^2, writes dL/dtheta to grad[49] and L to *loss.
 *   d_u, d_t: device float arrays of n entries; w: host float[65] in the order w1[16], b1[16],
 *   w2[16], b2, cap[16]; grad: host float[49] (the caps are fixed, not trained).
 *   Runs on `stream` and waits for it. Uses the current device.
 * Errors: PLANB_EINVAL (null pointer, n >= 2^32), PLANB_ENOMEM, PLANB_ECUDA.
 */
int planb_mlp_grad(const float *d_u, const float *d_t, size_t n, const float *w, float *grad,
                   double *loss, planb_stream_t stream);

/*
 * planb_mlp_grad_split — planb_mlp_grad on the two-float input the training uses: entry i of the
 * root's input is the unevaluated sum d_u[i] + d_ulo[i] (the range-reduced key carried to about
 * 48 bits), and the first layer adds the parts as the lookup's model evaluation does. Arguments and
 * errors as planb_mlp_grad; d_ulo is a device float array of n entries.
 */
int planb_mlp_grad_split(const float *d_u, const float *d_ulo, const float *d_t, size_t n,
                         const float *w, float *grad, double *loss, planb_stream_t stream);

/*
 * planb_mlp_knot_step — one iteration of the root's training loop as the table build runs it: the
 * full-batch gradient kernel, then the knot-value Adam kernel. The root is the linear spline
 * through the points (knots[h], v[h]), h = 0..16 (unit input weights, b1[h] = -knots[h], caps
 * knots[h+1] - knots[h] except the last unit's): w2[h] = (v[h+1] - v[h]) / (knots[h+1] - knots[h]),
 * b2 = v[0]. The kernel carries dL/dw2 and dL/db2 to dL/dv by the chain rule and applies Adam
 * (Kingma and Ba; beta1 0.9, beta2 0.999, eps 1e-8) to v.
 *   d_u, d_ulo (nullable: single-float input), d_t: device float arrays of n entries.
 *   w: host float[65] (w1, b1, w2, b2, cap), rewritten with the new w2 and b2; knots: host
 *   float[17]; v, m, q: host float[17] (knot values and Adam's two moments), rewritten; step: the
 *   steps already taken (this one is step + 1); lr: the learning rate; *loss: the loss before the
 *   update. Synchronous on `stream`; uses the current device. The paper has no learned part.
 * Errors: PLANB_EINVAL (null pointer, step < 0, n >= 2^32), PLANB_ENOMEM, PLANB_ECUDA.
 */
int planb_mlp_knot_step(const float *d_u, const float *d_ulo, const float *d_t, size_t n,
                        float *w, const float *knots, float *v, float *m, float *q, int32_t step,
                        float lr, double *loss, planb_stream_t stream);

/*
 * planb_mlp_forward — y(u) for every entry of the device array d_u (n floats) into d_y (device);
 * w (65 floats) as in planb_mlp_grad. Asynchronous on `stream`.
 * Errors: PLANB_EINVAL, PLANB_ECUDA.
 */
int planb_mlp_forward(const float *d_u, size_t n, const float *w, float *d_y,
                      planb_stream_t stream);

/* ------------------------------------------------------------------ host-only entry points */
/* These run on the host alone and need no GPU (except planb_intervals_device, the device
 * builder's counterpart of planb_intervals); they expose the build steps for inspection.     */

/*
 * planb_intervals — the elementary intervals of a prefix table (Section 3.1; Algorithm 2's event
 * sort and stack sweep, read as: exclusive range ends in 129-bit arithmetic, ends before starts at
 * one address, starts by ascending length, one interval per distinct boundary): out_start_hi/lo
 * receive the first address of each interval, strictly increasing from 0, and out_nh its next hop.
 * `cap` is the room in the output arrays; *out_m receives the interval count m (<= 2N + 1). When
 * cap < m nothing is written, *out_m is set and PLANB_EINVAL is returned.
 * merge_equal_nh as in planb_opts.
 */
int planb_intervals(const uint64_t *prefix_hi, const uint64_t *prefix_lo, const uint8_t *len,
                    const uint16_t *nexthop, size_t n, int merge_equal_nh, uint64_t *out_start_hi,
                    uint64_t *out_start_lo, uint16_t *out_nh, size_t cap, size_t *out_m);

/*
 * planb_intervals_device — planb_intervals computed by the device builder (PLANB_BUILDER_DEVICE:
 * GPU radix sorts and the bracket-matching scan that replaces Algorithm 2's stack) on the current
 * device; same arguments, same results. Host arrays in and out; device scratch is allocated and
 * freed inside the call. Errors: as planb_intervals, plus PLANB_ENODEV (no sm_103 device current),
 * PLANB_ENOMEM (device scratch), PLANB_ECUDA.
 */
int planb_intervals_device(const uint64_t *prefix_hi, const uint64_t *prefix_lo,
                           const uint8_t *len, const uint16_t *nexthop, size_t n,
                           int merge_equal_nh, uint64_t *out_start_hi, uint64_t *out_start_lo,
                           uint16_t *out_nh, size_t cap, size_t *out_m);

typedef struct {
    uint32_t keys_per_node;  /* k */
    uint32_t fanout;         /* b = k + 1 */
    uint32_t depth;          /* D: levels including the leaf level */
    uint32_t reserved;
    uint64_t n_keys;         /* keys to index */
    uint64_t internal_nodes; /* sum over the D - 1 internal levels of b^l */
    uint64_t leaf_capacity;  /* b^(D - 1) leaf nodes */
    uint64_t key_capacity;   /* k * b^(D - 1) */
    uint64_t level_start[16];/* level_start(l) = k (b^l - 1) / (b - 1), in keys (Section 3.2) */
} planb_layout_t;

/*
 * planb_layout_info — the linearized B+-tree arithmetic of Section 3.2 for k keys per node and
 * n_keys keys: the smallest depth whose leaf level holds n_keys keys, the level starts and the
 * capacities. depth_override > 0 forces that depth instead (for checking the capacity figures).
 * Errors: PLANB_EINVAL (k < 1, or a depth beyond 16 levels).
 */
int planb_layout_info(uint32_t keys_per_node, uint64_t n_keys, uint32_t depth_override,
                      planb_layout_t *out);

/*
 * planb_child_index — key index of the first key of child c of the j-th node on level d
 * (Section 3.2: child_start(d, j, c) = level_start(d + 1) + (j * b + c) * k). Host-only helper
 * exposed for checking the index arithmetic.
 */
uint64_t planb_child_index(uint32_t keys_per_node, uint32_t d, uint64_t j, uint32_t c);

/*
 * planb_debug_inject — test hook (the paper has no counterpart): makes the next table build fail
 * as if memory ran out, on the host (point = 1) or at device allocation (point = 2); 0 clears it.
 * It lets a test check that a failed planb_update leaves the previous table current and correct.
 * Errors: PLANB_EINVAL for another point.
 */
int planb_debug_inject(int point);

/*
 * planb_debug_table_dump — test hook (the paper has no counterpart): copies the current table's
 * device image to host memory `dst`: the node array(s) (F16HI: the high halves, then the low
 * halves), the top-of-tree index of the hybrid and learned kernels (16 bytes per entry, zero-padded
 * to 128 bytes) and the m next hops (u16). *out_bytes receives its size; with cap smaller (or dst
 * NULL) nothing is copied and PLANB_EINVAL is returned. Tables made by the two builders from the
 * same prefixes and options have identical images. Errors: PLANB_EINVAL, PLANB_ECUDA.
 */
int planb_debug_table_dump(const planb_fib *fib, void *dst, size_t cap, size_t *out_bytes);

/*
 * planb_debug_kernel_info — test hook (the paper has no counterpart): the CUDA function attributes
 * of the lookup kernel a table uses (multi != 0: its multi-table form), out6[0..5] = registers per
 * thread, max threads per block, max dynamic shared bytes, local (spill) bytes per thread, static
 * shared bytes, constant bytes. Errors: PLANB_EINVAL, PLANB_ECUDA.
 */
int planb_debug_kernel_info(const planb_fib *fib, int multi, int *out6);

/*
 * planb_lookup_host_noalloc — the lookup of planb_lookup_host for callers that must not allocate
 * device memory. The paper has no counterpart.
 *
 * Who needs it: a packet-forwarding thread (the data plane that hands bursts of destination
 * addresses to the lookup) cannot call cudaMalloc, because an allocation can block for a long time
 * (it may synchronise the device and takes the driver's allocator locks) while packets queue up
 * behind it; the same holds for a process whose device memory is already handed out by another
 * allocator's pool (a framework's caching allocator), where a private cudaMalloc can fail or
 * fragment that pool. planb_lookup_host would allocate its staging buffers on first use.
 *
 * How: addresses and results are staged through one fixed array of PLANB_NOALLOC_MAX_KEYS x 18
 * bytes (4.5 MiB) declared in the library as a __device__ variable, so every GPU that loads the
 * library holds it until the process exits. The call allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine. Its first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture. The address is kept per device for the rest of the process, which assumes
 * the device's primary context lives as long: do not call this after a cudaDeviceReset.
 *   addr_hi, addr_lo: host arrays of n uint64_t; out: host array of n uint16_t. The call copies
 *   them in, runs the lookup kernel and copies the results out on `stream`, and returns after the
 *   stream has finished them (synchronous). Pinned host buffers copy fastest.
 *   The array keeps the previous call's contents; nothing in it needs to start at zero, since each
 *   call writes the n entries it reads. Calls from any thread share the one array, so two calls
 *   that overlapped on the GPU would race on it: the library serialises them with a process-wide
 *   lock held until the call's copies and kernel are done, on success and on every failure.
 * Errors: PLANB_EINVAL (null pointer with n > 0, n > PLANB_NOALLOC_MAX_KEYS), PLANB_ECUDA.
 */
#define PLANB_NOALLOC_MAX_KEYS 262144
int planb_lookup_host_noalloc(const planb_fib *fib, const uint64_t *addr_hi,
                              const uint64_t *addr_lo, size_t n, uint16_t *out,
                              planb_stream_t stream);

/* planb_version — library version, (major << 16) | minor. */
uint32_t planb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PLANB_H */
