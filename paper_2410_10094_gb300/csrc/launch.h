// Host-side launchers of the library's kernels. Internal; the public ABI is include/stc.h.
#pragma once

#include "common.cuh"

namespace stc {

using u64 = unsigned long long;

// Kernels launched by the calling thread since the last take_launches() (for the stats).
void note_launch(unsigned n = 1);
unsigned take_launches();

// ------------------------------------------------------------------ scans (scan.cu)
// Exclusive prefix sums: out[0] = 0, out[i] = in[0] + ... + in[i-1], out[n] = total.
// `scratch` holds scan_scratch_elems(n) elements of the output type.
int64_t scan_scratch_elems(int64_t n);
cudaError_t scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* scratch, cudaStream_t s);
cudaError_t scan_u32_u64(const uint32_t* in, u64* out, int64_t n, u64* scratch, cudaStream_t s);
cudaError_t scan_u64(const u64* in, u64* out, int64_t n, u64* scratch, cudaStream_t s);
// scan_u32_u64 over the first min(*dn, nmax) elements, the count read on the device (the grid
// and scratch sized for nmax); out[min(*dn, nmax)] = total.
cudaError_t scan_u32_u64_dev(const uint32_t* in, u64* out, int64_t nmax, const unsigned* dn, u64* scratch,
                             cudaStream_t s);

// ------------------------------------------------------------------ preparation (prep.cu)
// Contract key of every entry (the LN key of the contract modes): keys[i] = ckey(i).
cudaError_t launch_linearize(const int32_t* coords, int64_t n, const KeyPlan& p, u64* keys,
                             uint32_t* status, int sms, cudaStream_t s);

// Counting sort of arbitrary keys in [0, k): count, then scatter through a cursor copy of
// the offsets. perm[pos] = input index.
cudaError_t launch_key_count(const u64* keys, int64_t n, u64 k, uint32_t* cnt, uint32_t* status,
                             int sms, cudaStream_t s);
cudaError_t launch_key_scatter(const u64* keys, int64_t n, u64 k, uint32_t* cursor, uint32_t* perm,
                               int sms, cudaStream_t s);

// Group Y by contract key (Section 4.2): histogram of ckey, then (after a scan) a scatter
// of each entry's free key and value into its key's run.
// nonempty (may be null): K/32 words, zeroed by the caller, receive the bitmap of the contract
// keys that have at least one Y entry.
cudaError_t launch_y_count(const int32_t* coords, int64_t n, const KeyPlan& p, uint32_t* cnt,
                           uint32_t* status, int sms, cudaStream_t s, uint32_t* nonempty = nullptr);
// yfk receives 32-bit free keys when key32 is set (F_Y < 2^32), 64-bit ones otherwise.
cudaError_t launch_y_scatter(const int32_t* coords, const double* vals, int64_t n, const KeyPlan& p,
                             uint32_t* cursor, void* yfk, bool key32, double* yv, int sms, cudaStream_t s);

// X entries whose contract key has a non-empty Y run ("survivors"), compacted, with the
// run they will read and the total product count P (Section 4.3).
struct Survivors {
  u64* fk;          // X free key
  uint32_t* ck;     // X contract key (kept only when per-segment runs are needed; may be null)
  uint32_t* ystart; // first slot of the matching Y run
  uint32_t* w;      // run length = products this entry makes
  double* v;        // X value
  unsigned* count;  // number of survivors (device counter)
};
// With gcnt non-null, also counts survivors per X free key.
// `nonempty` (K / 32 words of scratch, may be null) is used when K <= kNonemptyMaxKeys: a
// bitmap of the contract keys that have a Y run, held in shared memory by the survey so that
// rows without a run skip the lookup; built here from the runs unless nonempty_built (then
// launch_y_count built it).
constexpr u64 kNonemptyMaxKeys = 1ull << 18;
cudaError_t launch_x_survey(const int32_t* coords, const double* vals, int64_t n, const KeyPlan& p,
                            const uint32_t* yoff, u64 K, Survivors sv, u64* P, uint32_t* gcnt, uint32_t* status,
                            uint32_t* nonempty, int sms, cudaStream_t s, bool nonempty_built = false);

// Dense X (Y runs exist for most contract keys): count entries with a run per X free key
// and the products, then place them in group order straight from the input, without an
// intermediate survivor list.
struct GroupedX;
cudaError_t launch_x_count(const int32_t* coords, int64_t n, const KeyPlan& p, const uint32_t* yoff, u64* P,
                           uint32_t* gcnt, uint32_t* status, int sms, cudaStream_t s);
cudaError_t launch_x_scatter_dense(const int32_t* coords, const double* vals, int64_t n, const KeyPlan& p,
                                   const uint32_t* yoff, uint32_t* gcur, GroupedX gx, uint32_t* status, int sms,
                                   cudaStream_t s);

// A tensor in key form split into (free part / FL, free part % FL, contract digits): see
// keyed_split_kernel. K and F are the contract and free key spaces (K * F = prod(shape)).
struct KeySplit {
  u64 K, F, FL;
  int32_t m;
  int32_t trailing;  // contracted modes last (1) or first (0)
  int64_t csize[kMaxOrder];
};
cudaError_t launch_keyed_split(const u64* keys, int64_t n, const KeySplit& ks, int32_t* out, uint32_t* status,
                               int sms, cudaStream_t s);

// ------------------------------------------------------------------ dense ids (ids.cu)
// Distinct keys collected in an open-addressing table and numbered densely (Section 4.1.2).
// keys[slots] (all-ones = empty), flags[slots + 1] (flags[slots] = the all-ones key was
// seen), prefix[slots + 2] = exclusive scan of flags: the id of the key in slot h is
// prefix[h], the all-ones key's is prefix[slots], and prefix[slots + 1] = D, the number of
// distinct keys, which is also the id given to a key the table lacks.
struct IdTable {
  u64* keys;
  uint32_t* flags;
  uint32_t* prefix;
  u64 slots;  // a power of two >= 2n
};
uint64_t id_table_slots(int64_t n);
cudaError_t launch_id_insert_keys(const u64* keys, int64_t n, const IdTable& t, uint32_t* status, int sms,
                                  cudaStream_t s);
// Inserts the contract key of every coordinate row.
cudaError_t launch_id_insert_rows(const int32_t* coords, int64_t n, const KeyPlan& p, const IdTable& t,
                                  uint32_t* status, int sms, cudaStream_t s);
// Flags the occupied slots and scans them into prefix (scratch: scan_scratch_elems(slots + 1)).
cudaError_t launch_id_number(const IdTable& t, uint32_t* scratch, int sms, cudaStream_t s);
cudaError_t launch_id_lookup_keys(const u64* keys, int64_t n, const IdTable& t, uint32_t* ids, int sms,
                                  cudaStream_t s);
// out[i] = (free coordinates of row i, ascending mode order; id of its contract key), nf + 1
// int32 per row. fmask has bit j set for each free mode j.
cudaError_t launch_id_rewrite_rows(const int32_t* coords, int64_t n, const KeyPlan& p, uint32_t fmask, int nf,
                                   const IdTable& t, int32_t* out, uint32_t* status, int sms, cudaStream_t s);

// ------------------------------------------------------------------ one global table (global.cu)
struct GlobalTable {
  u64* keys;    // [cap], kEmpty64 when free
  double* vals; // [cap]
  u64 mask;     // cap - 1, cap a power of two
};
// Expansion with a merge-path split over the survivors' product prefix `wpre` (ns+1
// entries, wpre[ns] = P): every CTA takes an equal share of the P products. probe: lanes that
// probe the table together (1: each lane alone over slots; 4 or 8: tiles over buckets of that
// many slots).
cudaError_t launch_expand_global(const u64* wpre, int64_t ns, u64 P, Survivors sv, const u64* yfk,
                                 const double* yv, u64 FY, GlobalTable t, uint32_t* status, int sms,
                                 cudaStream_t s, int probe);
// The same with P and the survivor count read on the device (no host read between the survey
// and the expansion).
cudaError_t launch_expand_global_dev(const u64* wpre, const unsigned* dns, const u64* dP, Survivors sv, const u64* yfk,
                                     const double* yv, u64 FY, GlobalTable t, uint32_t* status, int sms,
                                     cudaStream_t s, int probe);
// Occupied slots -> COO output (coordinates decoded from the key).
cudaError_t launch_compact_global(GlobalTable t, const OutPlan& op, int32_t* coords, double* vals,
                                  u64 out_cap, u64* nz, uint32_t* status, int sms, cudaStream_t s);

// ------------------------------------------------------------------ per-group tables (grouped.cu)
constexpr int kMaxClasses = 5;

struct ClassShape {
  uint32_t slots;    // table slots in shared memory
  uint32_t threads;  // threads per CTA
};
extern const ClassShape kClassShapes32[];  // 32-bit local keys (F_Y < 2^32)
extern const ClassShape kClassShapes64[];  // 64-bit local keys
extern const int kNumClasses32;
extern const int kNumClasses64;

// X survivors in group order: the entries of X free key g are [goff[g], goff[g+1]).
struct GroupedX {
  uint32_t* ystart;
  uint32_t* w;
  double* v;
  uint32_t* ck;  // contract keys (dense-row accumulation only; may be null)
};

// Output of the binning pass.
struct Bins {
  int nclasses;
  u64 tmax[kMaxClasses];      // a group goes to the first class with t <= tmax
  uint32_t* list[kMaxClasses];
  uint32_t* count;            // [kMaxClasses + 4]: classes, overflow groups, stream, rank, stash
  // Bitmap-row accumulation (single contractions with per-segment runs): groups with
  // t >= dense_min go to the stream list (0) when B_g <= stream_cap and repeats are expected
  // to be few (2 B_g <= F_Y), else to the stash list (2) when B_g <= stash_cap, else to the
  // rank list (1). A streamed group's output bound is B_g itself.
  uint32_t* dense_list[3];    // null when not used
  u64 dense_min;
  u64 stream_cap;
  u64 stash_cap;
  uint32_t* huge_list;        // overflow groups, their table offsets and capacities
  u64* huge_off;
  u64* huge_cap;
  u64* huge_slots;            // total overflow-table slots
  u64* out_cap;               // sum over groups of min(B_g, F_Y): bound on the output size
  uint32_t* status;
};

// Output region of one problem of a batch.
struct BatchOut {
  u64 FY;
  u64 out_cap;
  int32_t* coords;
  double* vals;
  OutPlan op;  // a whole number of 8-byte words (copied word by word)
};
static_assert(sizeof(OutPlan) % 8 == 0, "OutPlan must be a whole number of 8-byte words");

struct GroupArgs {
  const uint32_t* goff;
  GroupedX gx;
  const void* yfk;  // Y free keys in contract-key order: uint32_t when F_Y < 2^32, else u64
  const double* yv;
  u64 FY;
  OutPlan op;
  int32_t* coords;
  double* vals;
  u64 out_cap;
  u64* nz;
  uint32_t* status;
  // Output regions and counters, one per problem (one entry for a single contraction). For
  // batches also the problem of each group and the group's X free key within that problem
  // (both null for a single contraction, where the group index is the X free key).
  const BatchOut* bout;
  u64* bnz;
  const uint32_t* gprob;
  const u64* gfk;
  // Non-null: yuniq[r] = 1 at the first entry r of every Y run whose free keys are all
  // different (run_unique_kernel). A group of one X entry over such a run has one product per
  // output, and the warp kernels write it as a scaled copy of the run without a table.
  const uint8_t* yuniq;
};

// Where one group's outputs go, resolved once per group.
struct OutTarget {
  u64 FY;        // Y free key space of the group's problem
  u64 zrow;      // output key of the group's row: fX * F_Y
  u64 base;      // first output position reserved for the group
  u64 cap;       // output capacity of the group's problem
  int32_t* coords;
  double* vals;
  u64* counter;  // the problem's output counter (positions are reserved from it)
  uint32_t prob; // problem whose output plan `op` holds (kNoProb before the first group)
  OutPlan op;
};
constexpr uint32_t kNoProb = 0xffffffffu;

// A count only the device knows (launchers then run a full persistent grid).
constexpr uint32_t kCountOnDevice = 0xffffffffu;

struct HugeGroups {
  uint32_t count;             // number of overflow groups, or kCountOnDevice
  const uint32_t* countp;     // device copy of the count, read by the kernel
  const uint32_t* list;
  const u64* off;
  const u64* cap;
  u64* keys;
  double* vals;
};

cudaError_t launch_x_group_scatter(Survivors sv, uint32_t* gcur, GroupedX gx, int64_t max_ns, int sms,
                                   cudaStream_t s);
cudaError_t launch_bin_groups(u64 FX, const uint32_t* goff, const uint32_t* gw, u64 FY, const Bins& b, int sms,
                              cudaStream_t s);
// direct: the shared-memory classes may write outputs as keys are first claimed (needs 32-bit
// keys and output positions below 2^32 in every problem). counts: host copies of the class
// counts (b.count), used to size the grids, or null when only the device knows them. depth:
// 0 the default expansion split of the direct CTA tables, 1 half as many products per lane
// per round.
cudaError_t launch_group_classes(const GroupArgs& a, bool wide_keys, bool direct, const Bins& b,
                                 const uint32_t* counts, int sms, cudaStream_t s, int depth = 0);
cudaError_t launch_group_huge(const GroupArgs& a, const HugeGroups& h, bool wide_keys, int sms, cudaStream_t s);

// ------------------------------------------------------------------ batches (batch.cu)
// One problem of a batch as the device kernels see it.
struct BatchProb {
  const int32_t* xc;
  const double* xv;
  const int32_t* yc;
  const double* yv;
  KeyPlan kx, ky;
  u64 koff;   // first contract-key bin of this problem in the concatenated bins
  u64 fxoff;  // offset of this problem's X free keys in the combined group-key space
  u64 FY;
};

// A probing table giving each distinct group key a number: its slot.
struct IdMap {
  u64* keys;  // [mask + 1], kEmpty64 when free
  u64 mask;
};

struct BatchArgs {
  int n;
  const BatchProb* pb;
  const int64_t* xrow;  // [n + 1] row offsets of X in the flattened row space
  const int64_t* yrow;  // [n + 1]
  const u64* fxoff;     // [n + 1]
  int64_t total_x, total_y;
  u64 bins;             // concatenated contract-key bins
  uint32_t* ycnt;
  uint32_t* yoff;       // [bins + 1]
  uint32_t* ycur;
  void* yfk;
  bool key32;
  double* yv;
  Survivors sv;
  u64* P;               // total products
  u64* Pp;              // [n] products per problem
  IdMap idmap;
  uint32_t* gid;        // [total_x] group number (table slot) of each survivor
  uint32_t* gcnt;       // [table size] survivors per group
  uint32_t* goff;       // [table size + 1]
  uint32_t* gcur;       // [table size]
  u64* pcap;            // [n] output bound per problem
  uint32_t* scan_scratch32;
  uint32_t* status;
  uint8_t* yuniq;       // [total_y] or null: runs with all-different free keys (32-bit keys only)
};

cudaError_t launch_batch_prepare(const BatchArgs& ba, int sms, cudaStream_t s);

// Where one run of a captured batch puts its outputs (written by the host before each replay).
struct BatchLayoutArgs {
  unsigned char* out;  // output block: values of every problem, then coordinates
  u64 out_bytes;       // its size
  u64* huge_keys;      // overflow groups' table
  double* huge_vals;
  u64 huge_cap;        // its slots
};
// Places every problem's output region in the run's block from the exact bounds pcap[n]
// (offs: [n + 1] value offsets, then [n + 1] coordinate offsets, in elements), then clears
// the slots of the overflow table this run uses (a grid of its own); flags kStatOutOverflow
// (and places nothing) when the block is too small.
cudaError_t launch_batch_layout(int n, const u64* pcap, const int32_t* oz, BatchOut* bo, const BatchLayoutArgs* args,
                                u64* offs, const u64* huge_slots, uint32_t* huge_count, uint32_t* status, int sms,
                                cudaStream_t s);
cudaError_t launch_batch_group(const BatchArgs& ba, GroupedX gx, const Bins& b, uint32_t* gprob, u64* gfk, int sms,
                               cudaStream_t s);

// Bitmap-row accumulation: each group's outputs are found one free-key segment at a time
// through a bitmap over the segment's free keys. `yoff` are the per-(contract key, segment)
// run offsets; seg is the segment width (a power of two, 64 <= seg <= kDenseSeg). Groups
// with at most dense_stash_cap() products (per segment) go to the stash kernel, the others
// to the rank kernel.
constexpr uint32_t kDenseSeg = 65536;
constexpr size_t kBitmapSmemPerCta = 112 * 1024;  // two CTAs per SM
uint32_t dense_stash_cap();

// Streamed bitmap rows: per group segment, its reservation and counts, for the hole filling
// that follows.
struct StreamRec {
  u64 base;           // first reserved position
  uint32_t firsts;    // outputs (first products), at [base, base + firsts)
  uint32_t products;  // reserved positions
};
struct StreamArgs {
  StreamRec* rec;
  unsigned* nrec;  // records: one per (streamed group, segment), [list position * nseg + segment]
  u64* holes;      // total repeats (positions that hold no output at the end)
};
// Lane-private dense rows for output rows of at most 64 free keys (FY <= 64, 32-bit Y free
// keys): one warp per group g in [0, ngroups) (empty groups skipped), outputs in key order.
cudaError_t launch_group_lanerow(const GroupArgs& a, u64 ngroups, uint32_t FY, int sms, cudaStream_t s);
uint32_t dense_stream_cap();
// Streamed groups (B_g <= dense_stream_cap()); launched after every other accumulation kernel.
// fixed_rows: the output plan has 2..8 modes in concatenation order, not all powers of two.
cudaError_t launch_group_stream(const GroupArgs& a, const uint32_t* yoff, uint32_t nseg, uint32_t seg,
                                const uint32_t* list, uint32_t count, StreamArgs sa, bool fixed_rows, int sms,
                                cudaStream_t s);
// Moves the entries above nnz into the holes below it.
// holes_total < 2^32 (positions above nnz are kept as 32-bit offsets).
cudaError_t launch_stream_fill(const StreamRec* rec, const unsigned* nrec, u64 nnz, u64 holes_total, uint32_t* src_pos,
                               u64* counters2, int32_t* coords, double* vals, int oz, uint32_t* status, int sms,
                               cudaStream_t s);
cudaError_t launch_group_dense(const GroupArgs& a, const uint32_t* yoff, uint32_t nseg, uint32_t seg,
                               const uint32_t* stash_list, uint32_t stash_count, const uint32_t* rank_list,
                               uint32_t rank_count, int sms, cudaStream_t s);

}  // namespace stc
