// TEST INFRASTRUCTURE -- a plain, slow CPU oracle for sparse COO tensor contraction
// (Swift, arXiv 2410.10094). Only the test suite, the smoke check and the benchmark's
// CPU-baseline leg may load or call this code; the library never does, and this file
// shares no code with the CUDA path.
//
// Each entry point writes out the definition, or the steps, of one passage of the paper:
//   oracle_contract        the contraction itself, Eq. 2 (Section 2.2)
//   oracle_ln_key          the "large number" (LN) key of a mode subset (Section 2.4.1, Fig. 3)
//   oracle_counting_sort   counting sort: count, cumulative sum, place (Section 4.1.1, Fig. 6)
//   oracle_first_seen_ids  small numbers assigned in order of first sight (Section 4.1.2, Fig. 7)
//   oracle_group_bounds    exact accumulation-table bound per X free group (Section 4.3)
//   oracle_table_slots     the x1.3 probing-table sizing rule (Section 2.3.1, Section 4.3)
//
// Floating point: FP64 throughout. The build passes -ffp-contract=off so that every
// product x*y is rounded before it is added (no fused multiply-add).
//
// Return codes: 0 ok, 1 invalid argument, 2 paired mode lengths differ,
// 3 coordinate out of range, 4 key does not fit in 64 bits.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

namespace {

enum { OK = 0, INVALID = 1, SHAPE_MISMATCH = 2, COORD_RANGE = 3, KEY_OVERFLOW = 4 };

struct Tensor {
  int32_t order;
  const int64_t* shape;
  int64_t nnz;
  const int32_t* coords;  // [nnz][order], row-major
  const double* vals;     // [nnz]
  int32_t at(int64_t i, int32_t mode) const { return coords[i * order + mode]; }
};

int check_tensor(const Tensor& t) {
  if (t.order < 0 || t.order > 64 || t.nnz < 0) return INVALID;
  if (t.nnz > 0 && (t.vals == nullptr || (t.order > 0 && t.coords == nullptr))) return INVALID;
  for (int32_t j = 0; j < t.order; j++)
    if (t.shape[j] < 1) return INVALID;
  for (int64_t i = 0; i < t.nnz; i++)
    for (int32_t j = 0; j < t.order; j++)
      if (t.at(i, j) < 0 || (int64_t)t.at(i, j) >= t.shape[j]) return COORD_RANGE;
  return OK;
}

// Modes of `order` that are not listed in `contracted`, in ascending order.
std::vector<int32_t> free_modes(int32_t order, const std::vector<int32_t>& contracted) {
  std::vector<int32_t> f;
  for (int32_t j = 0; j < order; j++) {
    bool c = false;
    for (int32_t k : contracted) c = c || (k == j);
    if (!c) f.push_back(j);
  }
  return f;
}

// Validates the contraction's mode lists: cx[i] pairs with cy[i] and both have the same
// length (Section 2.2: contracted modes must have equal lengths).
int check_pairs(const Tensor& X, const Tensor& Y, int32_t m, const int32_t* cx, const int32_t* cy,
                std::vector<int32_t>& vx, std::vector<int32_t>& vy) {
  if (m < 0 || m > X.order || m > Y.order) return INVALID;
  if (m > 0 && (cx == nullptr || cy == nullptr)) return INVALID;
  for (int32_t i = 0; i < m; i++) {
    if (cx[i] < 0 || cx[i] >= X.order || cy[i] < 0 || cy[i] >= Y.order) return INVALID;
    for (int32_t k = 0; k < i; k++)
      if (cx[k] == cx[i] || cy[k] == cy[i]) return INVALID;
    vx.push_back(cx[i]);
    vy.push_back(cy[i]);
  }
  for (int32_t i = 0; i < m; i++)
    if (X.shape[cx[i]] != Y.shape[cy[i]]) return SHAPE_MISMATCH;
  return OK;
}

struct Acc {
  double sum = 0.0;   // the output value: sum of x*y in the order the loops visit them
  double abs = 0.0;   // sum of |x*y|, the scale of the rounding error of any summation order
  int64_t cnt = 0;    // number of products that landed here
};

struct ContractResult {
  int32_t order = 0;
  uint64_t products = 0;
  std::vector<int32_t> coords;
  std::vector<double> vals, abs;
  std::vector<int64_t> cnt;
};

struct GroupResult {
  int32_t order = 0;  // number of X free modes
  uint64_t total = 0;
  std::vector<int32_t> coords;
  std::vector<uint64_t> bound;
  std::vector<int64_t> entries;
};

}  // namespace

extern "C" {

// Eq. 2: z[fX, fY] = sum over c of x[fX, c] * y[c, fY].
//
// Over COO lists this is: for every pair (x_i, y_j) whose contract coordinates agree
// (x's modes cx[0..m) against y's modes cy[0..m), pairwise), add x_i*y_j to the output
// entry whose coordinates are X's free coordinates (ascending mode order) followed by
// Y's free coordinates (ascending mode order). With `out_order`, output mode q holds
// that concatenation's entry out_order[q]. Repeated input coordinates are additive.
// Every output coordinate that received at least one product is kept, even when its
// value sums to 0.0. Output entries come out in lexicographic coordinate order.
//
// Y is first indexed by its contract tuple (an ordered map from tuple to the list of Y
// entries, in input order), so each x visits only its matching y's; summation order per
// output is x in input order, then y in input order.
int oracle_contract(int32_t ox, const int64_t* shx, int64_t nx, const int32_t* xc, const double* xv,
                    int32_t oy, const int64_t* shy, int64_t ny, const int32_t* yc, const double* yv,
                    int32_t m, const int32_t* cx, const int32_t* cy, const int32_t* out_order,
                    void** out) {
  if (out == nullptr) return INVALID;
  *out = nullptr;
  Tensor X{ox, shx, nx, xc, xv}, Y{oy, shy, ny, yc, yv};
  int rc = check_tensor(X);
  if (rc) return rc;
  rc = check_tensor(Y);
  if (rc) return rc;
  std::vector<int32_t> vcx, vcy;
  rc = check_pairs(X, Y, m, cx, cy, vcx, vcy);
  if (rc) return rc;
  std::vector<int32_t> xfree = free_modes(ox, vcx), yfree = free_modes(oy, vcy);
  const int32_t oz = (int32_t)(xfree.size() + yfree.size());
  if (out_order) {
    std::vector<int> seen(oz, 0);
    for (int32_t q = 0; q < oz; q++) {
      if (out_order[q] < 0 || out_order[q] >= oz || seen[out_order[q]]) return INVALID;
      seen[out_order[q]] = 1;
    }
  }

  std::map<std::vector<int32_t>, std::vector<int64_t>> y_by_contract;
  for (int64_t j = 0; j < ny; j++) {
    std::vector<int32_t> c(m);
    for (int32_t k = 0; k < m; k++) c[k] = Y.at(j, cy[k]);
    y_by_contract[c].push_back(j);
  }

  std::map<std::vector<int32_t>, Acc> z;
  uint64_t products = 0;
  std::vector<int32_t> c(m), cat(oz), zc(oz);
  for (int64_t i = 0; i < nx; i++) {
    for (int32_t k = 0; k < m; k++) c[k] = X.at(i, cx[k]);
    auto hit = y_by_contract.find(c);
    if (hit == y_by_contract.end()) continue;
    for (size_t a = 0; a < xfree.size(); a++) cat[a] = X.at(i, xfree[a]);
    for (int64_t j : hit->second) {
      for (size_t b = 0; b < yfree.size(); b++) cat[xfree.size() + b] = Y.at(j, yfree[b]);
      for (int32_t q = 0; q < oz; q++) zc[q] = out_order ? cat[out_order[q]] : cat[q];
      const double p = xv[i] * yv[j];
      Acc& acc = z[zc];
      acc.sum += p;
      acc.abs += std::fabs(p);
      acc.cnt += 1;
      products += 1;
    }
  }

  ContractResult* r = new ContractResult;
  r->order = oz;
  r->products = products;
  r->coords.reserve(z.size() * (size_t)oz);
  for (const auto& kv : z) {
    r->coords.insert(r->coords.end(), kv.first.begin(), kv.first.end());
    r->vals.push_back(kv.second.sum);
    r->abs.push_back(kv.second.abs);
    r->cnt.push_back(kv.second.cnt);
  }
  *out = r;
  return OK;
}

int64_t oracle_result_nnz(void* h) { return (int64_t)static_cast<ContractResult*>(h)->vals.size(); }
int32_t oracle_result_order(void* h) { return static_cast<ContractResult*>(h)->order; }
uint64_t oracle_result_products(void* h) { return static_cast<ContractResult*>(h)->products; }

void oracle_result_copy(void* h, int32_t* coords, double* vals, double* abs, int64_t* cnt) {
  const ContractResult* r = static_cast<ContractResult*>(h);
  if (coords && !r->coords.empty()) std::memcpy(coords, r->coords.data(), r->coords.size() * sizeof(int32_t));
  if (vals && !r->vals.empty()) std::memcpy(vals, r->vals.data(), r->vals.size() * sizeof(double));
  if (abs && !r->abs.empty()) std::memcpy(abs, r->abs.data(), r->abs.size() * sizeof(double));
  if (cnt && !r->cnt.empty()) std::memcpy(cnt, r->cnt.data(), r->cnt.size() * sizeof(int64_t));
}

void oracle_result_free(void* h) { delete static_cast<ContractResult*>(h); }

// The LN key (Section 2.4.1, Fig. 3): the coordinates of the listed modes read as the
// digits of one mixed-radix number, the first listed mode most significant and each
// digit's radix its mode's length. Fig. 3's two-mode example with length 10 maps (5, 1)
// to 51. Written in Horner form, key = (...(c0 * n1 + c1) * n2 + c2 ...).
int oracle_ln_key(int32_t order, const int64_t* shape, int64_t n, const int32_t* coords, int32_t k,
                  const int32_t* modes, uint64_t* keys_out) {
  if (order < 0 || n < 0 || k < 0 || k > order || (n > 0 && keys_out == nullptr)) return INVALID;
  for (int32_t t = 0; t < k; t++)
    if (modes[t] < 0 || modes[t] >= order) return INVALID;
  unsigned __int128 space = 1;
  for (int32_t t = 0; t < k; t++) {
    space *= (unsigned __int128)shape[modes[t]];
    if (space > (unsigned __int128)UINT64_MAX) return KEY_OVERFLOW;
  }
  for (int64_t i = 0; i < n; i++) {
    unsigned __int128 key = 0;
    for (int32_t t = 0; t < k; t++) {
      const int32_t c = coords[i * order + modes[t]];
      if (c < 0 || (int64_t)c >= shape[modes[t]]) return COORD_RANGE;
      key = key * (unsigned __int128)shape[modes[t]] + (unsigned __int128)c;
    }
    keys_out[i] = (uint64_t)key;
  }
  return OK;
}

// Counting sort (Section 4.1.1, Fig. 6) of n keys in [0, k): count each value, take the
// cumulative sum so that cum[v] is one past the last slot of value v, then walk the input
// and place each element at its value's pointer, decrementing the pointer. Walking from
// the last element to the first keeps equal keys in input order.
//   offsets_out[k+1]: offsets_out[v] is the first slot of value v, offsets_out[k] = n
//   perm_out[n]:      perm_out[s] is the input index placed at slot s
int oracle_counting_sort(int64_t n, const uint64_t* keys, uint64_t k, int64_t* offsets_out,
                         int64_t* perm_out) {
  if (n < 0 || offsets_out == nullptr || (n > 0 && (keys == nullptr || perm_out == nullptr))) return INVALID;
  std::vector<int64_t> count(k, 0);
  for (int64_t i = 0; i < n; i++) {
    if (keys[i] >= k) return COORD_RANGE;
    count[keys[i]] += 1;
  }
  std::vector<int64_t> cum(k, 0);
  int64_t run = 0;
  for (uint64_t v = 0; v < k; v++) {
    run += count[v];
    cum[v] = run;
    offsets_out[v] = run - count[v];
  }
  offsets_out[k] = run;
  for (int64_t i = n - 1; i >= 0; i--) {
    cum[keys[i]] -= 1;
    perm_out[cum[keys[i]]] = i;
  }
  return OK;
}

// Small numbers (Section 4.1.2, Fig. 7): scan the keys in order; a key already in the
// table gets its stored number, a new key gets the number of keys stored so far.
int oracle_first_seen_ids(int64_t n, const uint64_t* keys, int64_t* ids_out, int64_t* ndistinct) {
  if (n < 0 || ndistinct == nullptr || (n > 0 && (keys == nullptr || ids_out == nullptr))) return INVALID;
  std::map<uint64_t, int64_t> table;
  for (int64_t i = 0; i < n; i++) {
    auto it = table.find(keys[i]);
    if (it != table.end()) {
      ids_out[i] = it->second;
    } else {
      const int64_t id = (int64_t)table.size();
      table.emplace(keys[i], id);
      ids_out[i] = id;
    }
  }
  *ndistinct = (int64_t)table.size();
  return OK;
}

// Exact accumulation-table bound (Section 4.3): the X entries that share a free tuple form
// one group; each entry will meet exactly count_Y[its contract tuple] Y entries, so the
// group's output entries number at most the sum of those counts. The total over groups is
// the number of products P. Groups come out in lexicographic order of the X free tuple.
int oracle_group_bounds(int32_t ox, const int64_t* shx, int64_t nx, const int32_t* xc,
                        int32_t oy, const int64_t* shy, int64_t ny, const int32_t* yc,
                        int32_t m, const int32_t* cx, const int32_t* cy, void** out) {
  if (out == nullptr) return INVALID;
  *out = nullptr;
  static const double kUnused = 0.0;
  Tensor X{ox, shx, nx, xc, &kUnused}, Y{oy, shy, ny, yc, &kUnused};
  int rc = check_tensor(X);
  if (rc) return rc;
  rc = check_tensor(Y);
  if (rc) return rc;
  std::vector<int32_t> vcx, vcy;
  rc = check_pairs(X, Y, m, cx, cy, vcx, vcy);
  if (rc) return rc;
  std::vector<int32_t> xfree = free_modes(ox, vcx);

  std::map<std::vector<int32_t>, uint64_t> count_y;
  for (int64_t j = 0; j < ny; j++) {
    std::vector<int32_t> c(m);
    for (int32_t k = 0; k < m; k++) c[k] = Y.at(j, cy[k]);
    count_y[c] += 1;
  }
  std::map<std::vector<int32_t>, std::pair<uint64_t, int64_t>> groups;
  uint64_t total = 0;
  for (int64_t i = 0; i < nx; i++) {
    std::vector<int32_t> c(m), f(xfree.size());
    for (int32_t k = 0; k < m; k++) c[k] = X.at(i, cx[k]);
    for (size_t a = 0; a < xfree.size(); a++) f[a] = X.at(i, xfree[a]);
    auto it = count_y.find(c);
    const uint64_t w = (it == count_y.end()) ? 0 : it->second;
    auto& g = groups[f];
    g.first += w;
    g.second += 1;
    total += w;
  }
  GroupResult* r = new GroupResult;
  r->order = (int32_t)xfree.size();
  r->total = total;
  for (const auto& kv : groups) {
    r->coords.insert(r->coords.end(), kv.first.begin(), kv.first.end());
    r->bound.push_back(kv.second.first);
    r->entries.push_back(kv.second.second);
  }
  *out = r;
  return OK;
}

int64_t oracle_groups_count(void* h) { return (int64_t)static_cast<GroupResult*>(h)->bound.size(); }
int32_t oracle_groups_order(void* h) { return static_cast<GroupResult*>(h)->order; }
uint64_t oracle_groups_total(void* h) { return static_cast<GroupResult*>(h)->total; }

void oracle_groups_copy(void* h, int32_t* coords, uint64_t* bound, int64_t* entries) {
  const GroupResult* r = static_cast<GroupResult*>(h);
  if (coords && !r->coords.empty()) std::memcpy(coords, r->coords.data(), r->coords.size() * sizeof(int32_t));
  if (bound && !r->bound.empty()) std::memcpy(bound, r->bound.data(), r->bound.size() * sizeof(uint64_t));
  if (entries && !r->entries.empty()) std::memcpy(entries, r->entries.data(), r->entries.size() * sizeof(int64_t));
}

void oracle_groups_free(void* h) { delete static_cast<GroupResult*>(h); }

// Probing tables are commonly made 1.3 times the largest number of entries they must hold
// (Section 2.3.1); the Section 4.3 example turns a bound of 7 into 9 slots, i.e. the
// integer part of 1.3 * bound.
uint64_t oracle_table_slots(uint64_t bound) { return (uint64_t)std::floor(1.3 * (double)bound); }

}  // extern "C"
