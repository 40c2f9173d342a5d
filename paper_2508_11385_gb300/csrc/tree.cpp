// tree.cpp -- validation, canonicalisation, kernel choice and code generation.
//
// A coot_tree is the run-time form of the paper's expression types (Sec. 3):
// leaves are Mat objects, N_TRANS is Op<T1,op_trans>, the unary and scalar
// kinds are eOp<T1,eop_type>, N_PLUS..N_DIV are eGlue<T1,T2,eglue_type>.
// As with Bandicoot's compile-time pattern matching, the whole tree is
// analysed before anything runs:
//   - shapes are checked as Armadillo does ("incompatible matrix dimensions");
//   - trans() is pushed down to the leaves -- trans(A + B) reads A and B
//     transposed -- so a transpose never materialises (the paper's implicit
//     transpose of trans(X)*Y, applied to element-wise trees);
//   - identical leaf reads are merged, so every distinct operand element is
//     loaded once;
//   - the tree is spelt as a C++ type over the device expression templates,
//     which NVRTC instantiates into one kernel per tree (Sec. 4 notes that
//     Bandicoot otherwise chains predefined kernels; fusing the tree into one
//     generated kernel is the follow-up the conclusion announces).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <array>
#include <map>
#include <sstream>
#include <tuple>

#include "coot_internal.h"

namespace cg {

const char* family_name(Family f) {
  switch (f) {
    case F_STR: return "str";
    case F_COL: return "col";
    case F_ROW: return "row";
    case F_TILE: return "tile";
    case F_ADJ: return "adj";
    case F_BATCH: return "batch";
    case F_SCAN: return "scan";
    case F_GEMM: return "gemm";
  }
  return "?";
}

static int esize(int32_t d) {
  switch (d) {
    case COOT_F32: return 4;
    case COOT_F64: return 8;
    case COOT_BF16: return 2;
    case COOT_F16: return 2;
    case COOT_I32: return 4;
  }
  return 0;
}

std::string storage_type_name(coot_dtype d) {
  switch (d) {
    case COOT_F32: return "float";
    case COOT_F64: return "double";
    case COOT_BF16: return "bf16";
    case COOT_F16: return "f16";
    case COOT_I32: return "int";
  }
  return "?";
}

static bool is_unary(int op) {
  return op == COOT_N_NEG || op == COOT_N_EXP || op == COOT_N_LOG || op == COOT_N_ABS || op == COOT_N_SQUARE ||
         op == COOT_N_SQRT;
}
static bool is_scalar_op(int op) { return op >= COOT_N_SCAL_TIMES && op <= COOT_N_SCAL_DIV_POST; }
static bool is_binary(int op) { return op >= COOT_N_PLUS && op <= COOT_N_DIV; }

static int64_t mat_rs(const coot_mat& m) { return m.rs > 1 ? m.rs : 1; }

static bool mat_shape_ok(const coot_mat& m) {
  if (m.n_rows < 0 || m.n_cols < 0 || m.rs < 0) return false;
  if (m.n_cols > 1 && m.ld < (m.n_rows > 0 ? (m.n_rows - 1) * mat_rs(m) + 1 : 0)) return false;
  if (m.n_cols > 1 && m.ld < 1) return false;
  return true;
}

static int64_t mat_ld(const coot_mat& m) { return (m.n_cols > 1) ? m.ld : (m.ld > 0 ? m.ld : m.n_rows); }

// byte range [lo, hi) touched by nr x nc elements at base + (off + i*rs + j*cs)*esz
static void strided_range(const void* data, int64_t off, int64_t rs, int64_t cs, int64_t nr, int64_t nc, int esz,
                          uintptr_t* lo, uintptr_t* hi) {
  if (nr <= 0 || nc <= 0) {
    *lo = *hi = 0;
    return;
  }
  uintptr_t base = (uintptr_t)data;
  *lo = base + (uintptr_t)(off * esz);
  *hi = base + (uintptr_t)((off + (nr - 1) * rs + (nc - 1) * cs + 1) * esz);
}

coot_status analyse(const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves, const coot_mat* out,
                    coot_reduce red, Analysis* an) {
  *an = Analysis();
  if (!tree || !tree->nodes) return set_error(COOT_ERR_INVALID, "tree or tree->nodes is NULL");
  const int nn = tree->n_nodes;
  if (nn < 1 || nn > COOT_MAX_NODES) return set_error(COOT_ERR_INVALID, "n_nodes %d outside 1..%d", nn, COOT_MAX_NODES);
  if (!leaves || n_leaves < 1 || n_leaves > COOT_MAX_LEAVES)
    return set_error(COOT_ERR_INVALID, "n_leaves %d outside 1..%d (or leaves NULL)", n_leaves, COOT_MAX_LEAVES);
  const int32_t dt = leaves[0].dtype;
  if (esize(dt) == 0) return set_error(COOT_ERR_DTYPE, "leaf 0: unknown dtype %d", dt);
  for (int i = 0; i < n_leaves; ++i) {
    if (leaves[i].dtype != dt) return set_error(COOT_ERR_DTYPE, "leaf %d: all leaves must share one dtype", i);
    if (!mat_shape_ok(leaves[i]))
      return set_error(COOT_ERR_INVALID, "leaf %d: bad shape %lld x %lld, ld %lld", i, (long long)leaves[i].n_rows,
                       (long long)leaves[i].n_cols, (long long)leaves[i].ld);
    if (!leaves[i].data && leaves[i].n_rows * leaves[i].n_cols > 0)
      return set_error(COOT_ERR_INVALID, "leaf %d: NULL data", i);
  }
  an->dtype = (coot_dtype)dt;
  an->esz = esize(dt);
  an->ct = (dt == COOT_F64) ? CT_F64 : (dt == COOT_I32 ? CT_I32 : CT_F32);
  const bool is_int = (an->ct == CT_I32);
  // FP32 accumulation mode (float-float unless $COOT_ACCUM selects the
  // Kahan or plain variant for an accuracy comparison)
  if (an->ct == CT_F32) {
    const char* am = getenv("COOT_ACCUM");
    if (am && !strcmp(am, "kahan")) an->accum = 1;
    if (am && !strcmp(am, "plain")) an->accum = 2;
  }

  // ---- per-node checks and shape inference
  std::vector<int64_t> R(nn), Cc(nn);
  for (int n = 0; n < nn; ++n) {
    const coot_node& d = tree->nodes[n];
    const int op = d.op;
    if (op < 0 || op >= COOT_N_COUNT_) return set_error(COOT_ERR_INVALID, "node %d: unknown op %d", n, op);
    auto operand = [&](int idx, const char* nm) -> coot_status {
      if (idx < 0 || idx >= n)
        return set_error(COOT_ERR_INVALID, "node %d: operand %s = %d must refer to an earlier node", n, nm, idx);
      return COOT_OK;
    };
    coot_status s;
    if (op == COOT_N_LEAF) {
      if (d.leaf < 0 || d.leaf >= n_leaves) return set_error(COOT_ERR_INVALID, "node %d: leaf %d not given", n, d.leaf);
      R[n] = leaves[d.leaf].n_rows;
      Cc[n] = leaves[d.leaf].n_cols;
    } else if (op == COOT_N_SUBMAT) {
      if ((s = operand(d.a, "a"))) return s;
      if (tree->nodes[d.a].op != COOT_N_LEAF)
        return set_error(COOT_ERR_INVALID, "node %d: submat must view a leaf node", n);
      if (d.r0 < 0 || d.c0 < 0 || d.nr < 0 || d.nc < 0 || d.r0 + d.nr > R[d.a] || d.c0 + d.nc > Cc[d.a])
        return set_error(COOT_ERR_SHAPE, "node %d: submat (%lld,%lld) %lldx%lld outside %lldx%lld", n, (long long)d.r0,
                         (long long)d.c0, (long long)d.nr, (long long)d.nc, (long long)R[d.a], (long long)Cc[d.a]);
      R[n] = d.nr;
      Cc[n] = d.nc;
    } else if (op == COOT_N_TRANS) {
      if ((s = operand(d.a, "a"))) return s;
      R[n] = Cc[d.a];
      Cc[n] = R[d.a];
    } else if (op == COOT_N_EACH_COL) {
      if ((s = operand(d.a, "a"))) return s;
      if (Cc[d.a] != 1 || d.nc < 0)
        return set_error(COOT_ERR_SHAPE, "node %d: each_col repeats a column vector (operand is %lldx%lld, nc %lld)", n,
                         (long long)R[d.a], (long long)Cc[d.a], (long long)d.nc);
      R[n] = R[d.a];
      Cc[n] = d.nc;
    } else if (op == COOT_N_EACH_ROW) {
      if ((s = operand(d.a, "a"))) return s;
      if (R[d.a] != 1 || d.nr < 0)
        return set_error(COOT_ERR_SHAPE, "node %d: each_row repeats a row vector (operand is %lldx%lld, nr %lld)", n,
                         (long long)R[d.a], (long long)Cc[d.a], (long long)d.nr);
      R[n] = d.nr;
      Cc[n] = Cc[d.a];
    } else if (op == COOT_N_DIAG) {
      if ((s = operand(d.a, "a"))) return s;
      const int64_t k = d.r0;
      const int64_t len = (k >= 0) ? std::min(R[d.a], Cc[d.a] - k) : std::min(R[d.a] + k, Cc[d.a]);
      if (len < 0 || (k != 0 && (k >= Cc[d.a] || -k >= R[d.a])))
        return set_error(COOT_ERR_SHAPE, "node %d: diagonal %lld outside a %lldx%lld matrix", n, (long long)k,
                         (long long)R[d.a], (long long)Cc[d.a]);
      R[n] = std::max<int64_t>(len, 0);
      Cc[n] = 1;
    } else if (is_unary(op) || is_scalar_op(op)) {
      if ((s = operand(d.a, "a"))) return s;
      if (is_int && (op == COOT_N_EXP || op == COOT_N_LOG || op == COOT_N_SQRT))
        return set_error(COOT_ERR_DTYPE, "node %d: exp/log/sqrt are not defined for INT32 trees", n);
      if (is_scalar_op(op)) {
        if (is_int && !(std::isfinite(d.k) && d.k > -2147483649.0 && d.k < 2147483648.0))
          return set_error(COOT_ERR_INVALID, "node %d: scalar %g does not fit INT32", n, d.k);
      }
      R[n] = R[d.a];
      Cc[n] = Cc[d.a];
    } else if (is_binary(op)) {
      if ((s = operand(d.a, "a")) || (s = operand(d.b, "b"))) return s;
      if (R[d.a] != R[d.b] || Cc[d.a] != Cc[d.b])
        return set_error(COOT_ERR_SHAPE, "node %d: incompatible matrix dimensions: %lldx%lld and %lldx%lld", n,
                         (long long)R[d.a], (long long)Cc[d.a], (long long)R[d.b], (long long)Cc[d.b]);
      R[n] = R[d.a];
      Cc[n] = Cc[d.a];
    }
  }
  const int root = nn - 1;
  an->nr = R[root];
  an->nc = Cc[root];
  an->root_op = tree->nodes[root].op;

  // ---- reduction
  an->red = red;
  switch (red.kind) {
    case COOT_R_NONE: an->red_mode = RED_NONE; break;
    case COOT_R_ACCU: an->red_mode = RED_SUM; an->red.dim = -1; break;
    case COOT_R_SUM:
    case COOT_R_MEAN:
      if (red.dim < -1 || red.dim > 1) return set_error(COOT_ERR_INVALID, "reduction dim %d not in {-1,0,1}", red.dim);
      an->red_mode = RED_SUM;
      break;
    case COOT_R_DOT:
      if (an->root_op != COOT_N_SCHUR) return set_error(COOT_ERR_INVALID, "R_DOT needs a root node a %% b");
      an->red_mode = RED_DOT;
      an->red.dim = -1;
      break;
    case COOT_R_NORM2:
      if (an->nr != 1 && an->nc != 1)
        return set_error(COOT_ERR_SHAPE, "R_NORM2 is the vector 2-norm; use R_NORM_FRO for a %lldx%lld matrix",
                         (long long)an->nr, (long long)an->nc);
      an->red_mode = RED_SSQ;
      an->red.dim = -1;
      break;
    case COOT_R_NORM_FRO: an->red_mode = RED_SSQ; an->red.dim = -1; break;
    case COOT_R_VAR:
    case COOT_R_STDDEV:
      if (red.norm_type != 0 && red.norm_type != 1)
        return set_error(COOT_ERR_INVALID, "var/stddev norm_type must be 0 or 1");
      if (red.dim < -1 || red.dim > 1) return set_error(COOT_ERR_INVALID, "reduction dim %d not in {-1,0,1}", red.dim);
      an->red_mode = RED_CSQ;
      break;
    case COOT_R_MIN:
    case COOT_R_MAX:
    case COOT_R_INDEX_MIN:
    case COOT_R_INDEX_MAX:
    case COOT_R_PROD:
      if (red.dim < -1 || red.dim > 1) return set_error(COOT_ERR_INVALID, "reduction dim %d not in {-1,0,1}", red.dim);
      an->red_mode = red.kind == COOT_R_MIN         ? RED_MIN
                     : red.kind == COOT_R_MAX       ? RED_MAX
                     : red.kind == COOT_R_INDEX_MIN ? RED_IMIN
                     : red.kind == COOT_R_INDEX_MAX ? RED_IMAX
                                                    : RED_PROD;
      break;
    case COOT_R_CUMSUM:
      if (red.dim < -1 || red.dim > 1) return set_error(COOT_ERR_INVALID, "cumsum dim %d not in {-1,0,1}", red.dim);
      if (!out) return set_error(COOT_ERR_INVALID, "cumsum writes its result to out, which is NULL");
      if (red.dim == -1) an->red.dim = (an->nr == 1) ? 1 : 0;  // along a row vector, else down the columns
      an->red_mode = RED_NONE;
      break;
    default: return set_error(COOT_ERR_INVALID, "unknown reduction kind %d", red.kind);
  }
  if (is_int && (red.kind == COOT_R_MEAN || red.kind == COOT_R_NORM2 || red.kind == COOT_R_NORM_FRO ||
                 red.kind == COOT_R_VAR || red.kind == COOT_R_STDDEV))
    return set_error(COOT_ERR_DTYPE, "mean/norm/var/stddev are not defined for INT32 trees");
  if (red.n_seg < 0) return set_error(COOT_ERR_INVALID, "n_seg %d is negative", red.n_seg);
  if (red.n_seg > 1) {
    const bool along_rows = an->red.dim == 1 && red.kind != COOT_R_ACCU && red.kind != COOT_R_DOT &&
                            red.kind != COOT_R_NORM2 && red.kind != COOT_R_NORM_FRO && red.kind != COOT_R_NONE;
    if (!along_rows) return set_error(COOT_ERR_INVALID, "n_seg > 1 segments a reduction or cumsum along dim 1");
    if (an->nc % red.n_seg)
      return set_error(COOT_ERR_SHAPE, "n_seg %d does not divide the %lld columns", red.n_seg, (long long)an->nc);
  }
  an->red.n_seg = red.n_seg > 1 ? red.n_seg : 1;

  // ---- canonical form: push trans(), each_col / each_row and diag() down to
  // the leaf reads.  The state carried down is the affine map from the root's
  // element (i,j) to the current node's element (row, col):
  //   row = m[0] i + m[1] j + m[2],   col = m[3] i + m[4] j + m[5]
  // trans swaps the two lines, each_col sets col = 0, each_row sets row = 0,
  // diag(k) maps (row, 0) to (row + max(-k,0), row + max(k,0)).
  typedef std::array<int64_t, 6> Map;
  std::map<std::pair<int, Map>, int> memo;
  std::map<std::tuple<int, int64_t, int64_t, int64_t, int>, int> slot_of;
  std::function<int(int, const Map&)> canon = [&](int n, const Map& m) -> int {
    auto key = std::make_pair(n, m);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    const coot_node& d = tree->nodes[n];
    CNode c;
    if (d.op == COOT_N_LEAF || d.op == COOT_N_SUBMAT) {
      const int leaf = (d.op == COOT_N_LEAF) ? d.leaf : tree->nodes[d.a].leaf;
      const coot_mat& L = leaves[leaf];
      const int64_t r0 = (d.op == COOT_N_SUBMAT) ? d.r0 : 0, c0 = (d.op == COOT_N_SUBMAT) ? d.c0 : 0;
      const int64_t lrs = mat_rs(L), lld = mat_ld(L);
      int64_t rs = m[0] * lrs + m[3] * lld, cs = m[1] * lrs + m[4] * lld;
      const int64_t off = (m[2] + r0) * lrs + (m[5] + c0) * lld;
      // a transposed view of a leaf with adjacent rows goes through the tile
      // staging (whatever the shape, so that problems of a batch agree);
      // adjacent rows are direct; anything else is general
      const bool tr = (m[0] == 0 && m[1] == 1 && m[3] == 1 && m[4] == 0 && lrs == 1);
      if (!tr) {
        // a stride along an extent of one is never used: a single row reads
        // as adjacent rows, a single column as a contiguous one
        if (an->nr <= 1) rs = 1;
        if (an->nc <= 1) cs = an->nr;
      }
      const int kind = tr ? 1 : (rs == 1 ? 0 : 2);
      auto sk = std::make_tuple(leaf, off, rs, cs, kind);
      auto si = slot_of.find(sk);
      int sidx;
      if (si == slot_of.end()) {
        sidx = (int)an->slots.size();
        Slot sl;
        sl.leaf = leaf;
        sl.off = off;
        sl.rs = rs;
        sl.cs = cs;
        sl.trans = (kind == 1);
        sl.gen = (kind == 2);
        sl.r0 = m[2] + r0;  // trans: view origin (row, col) = (r0 + m2, c0 + m5)
        sl.c0 = m[5] + c0;
        sl.vr = an->nc;     // trans: view rows = tree columns
        sl.vc = an->nr;
        sl.full = (kind == 0 && off == 0 && lrs == 1 && an->nr == L.n_rows && an->nc == L.n_cols &&
                   (an->nc <= 1 || cs == lld));
        sl.n_distinct = (rs != 0 ? an->nr : 1) * (cs != 0 ? an->nc : 1);
        an->slots.push_back(sl);
        slot_of[sk] = sidx;
      } else {
        sidx = si->second;
      }
      c.op = COOT_N_LEAF;
      c.slot = sidx;
    } else if (d.op == COOT_N_TRANS) {
      int r = canon(d.a, Map{m[3], m[4], m[5], m[0], m[1], m[2]});
      memo[key] = r;
      return r;
    } else if (d.op == COOT_N_EACH_COL) {
      int r = canon(d.a, Map{m[0], m[1], m[2], 0, 0, 0});
      memo[key] = r;
      return r;
    } else if (d.op == COOT_N_EACH_ROW) {
      int r = canon(d.a, Map{0, 0, 0, m[3], m[4], m[5]});
      memo[key] = r;
      return r;
    } else if (d.op == COOT_N_DIAG) {
      const int64_t k = d.r0, kr = k < 0 ? -k : 0, kc = k > 0 ? k : 0;
      int r = canon(d.a, Map{m[0], m[1], m[2] + kr, m[0], m[1], m[2] + kc});
      memo[key] = r;
      return r;
    } else if (is_unary(d.op) || is_scalar_op(d.op)) {
      c.op = d.op;
      c.a = canon(d.a, m);
      if (is_scalar_op(d.op)) {
        c.kidx = (int)an->scalars.size();
        an->scalars.push_back(d.k);
      }
    } else {
      c.op = d.op;
      c.a = canon(d.a, m);
      c.b = canon(d.b, m);
    }
    int idx = (int)an->cn.size();
    an->cn.push_back(c);
    memo[key] = idx;
    return idx;
  };
  an->root = canon(root, Map{1, 0, 0, 0, 1, 0});
  if ((int)an->slots.size() > COOT_MAX_SLOTS)
    return set_error(COOT_ERR_UNSUPPORTED, "tree reads %d distinct leaf views; at most %d", (int)an->slots.size(),
                     COOT_MAX_SLOTS);
  if ((int)an->scalars.size() > COOT_MAX_SCALARS_DEV)
    return set_error(COOT_ERR_UNSUPPORTED, "tree has %d scalars; at most %d", (int)an->scalars.size(),
                     COOT_MAX_SCALARS_DEV);
  for (size_t s = 0; s < an->slots.size(); ++s) {
    if (an->slots[s].trans) {
      an->any_trans = true;
      an->trmask |= (1 << s);
    }
    if (an->slots[s].gen) an->gmask |= (1 << s);
  }
  if (an->n_seg() > 1 && an->any_trans && !an->scan())
    return set_error(COOT_ERR_UNSUPPORTED, "segmented reductions of trees with transposed reads are not implemented");

  // ---- C++ type of the canonical tree
  std::function<std::string(int)> spell = [&](int i) -> std::string {
    const CNode& c = an->cn[i];
    char buf[64];
    if (c.op == COOT_N_LEAF) {
      snprintf(buf, sizeof buf, "Leaf<%d>", c.slot);
      return buf;
    }
    const char* eop = nullptr;
    switch (c.op) {
      case COOT_N_NEG: eop = "eop_neg"; break;
      case COOT_N_EXP: eop = "eop_exp"; break;
      case COOT_N_LOG: eop = "eop_log"; break;
      case COOT_N_ABS: eop = "eop_abs"; break;
      case COOT_N_SQUARE: eop = "eop_square"; break;
      case COOT_N_SQRT: eop = "eop_sqrt"; break;
      default: break;
    }
    if (eop) return "eOp<" + spell(c.a) + ", " + eop + ">";
    const char* sop = nullptr;
    switch (c.op) {
      case COOT_N_SCAL_TIMES: sop = "eop_scalar_times"; break;
      case COOT_N_SCAL_PLUS: sop = "eop_scalar_plus"; break;
      case COOT_N_SCAL_MINUS_PRE: sop = "eop_scalar_minus_pre"; break;
      case COOT_N_SCAL_MINUS_POST: sop = "eop_scalar_minus_post"; break;
      case COOT_N_SCAL_DIV_PRE: sop = "eop_scalar_div_pre"; break;
      case COOT_N_SCAL_DIV_POST: sop = "eop_scalar_div_post"; break;
      default: break;
    }
    if (sop) {
      snprintf(buf, sizeof buf, "%s<%d>", sop, c.kidx);
      return "eOp<" + spell(c.a) + ", " + buf + ">";
    }
    const char* gop = nullptr;
    switch (c.op) {
      case COOT_N_PLUS: gop = "eglue_plus"; break;
      case COOT_N_MINUS: gop = "eglue_minus"; break;
      case COOT_N_SCHUR: gop = "eglue_schur"; break;
      case COOT_N_DIV: gop = "eglue_div"; break;
      default: break;
    }
    return "eGlue<" + spell(c.a) + ", " + spell(c.b) + ", " + gop + ">";
  };
  an->type_str = spell(an->root);

  // ---- output
  if (out) {
    an->has_out = true;
    if (out->dtype != dt) return set_error(COOT_ERR_DTYPE, "out dtype %d differs from the leaves' %d", out->dtype, dt);
    if (out->n_rows != an->nr || out->n_cols != an->nc)
      return set_error(COOT_ERR_SHAPE, "out is %lldx%lld, the tree is %lldx%lld", (long long)out->n_rows,
                       (long long)out->n_cols, (long long)an->nr, (long long)an->nc);
    if (!mat_shape_ok(*out)) return set_error(COOT_ERR_INVALID, "out: bad ld or row stride");
    if (!out->data && an->nr * an->nc > 0) return set_error(COOT_ERR_INVALID, "out: NULL data");
    an->out_rs = mat_rs(*out);
    if (an->out_rs != 1 && an->nr > 1) an->gmask |= (1 << COOT_MAX_SLOTS);
    return check_out_alias(*an, leaves, out);
  }
  return COOT_OK;
}

// aliasing: overlap of out with a leaf read is allowed only for an identical
// read (same elements in the same order: each element is read and written by
// one thread)
coot_status check_out_alias(const Analysis& an, const coot_mat* leaves, const coot_mat* out) {
  if (!out) return COOT_OK;
  const int64_t ocs = an.nc > 1 ? mat_ld(*out) : 0, ors = an.nr > 1 ? an.out_rs : 0;
  uintptr_t olo, ohi;
  strided_range(out->data, 0, an.out_rs, mat_ld(*out), an.nr, an.nc, an.esz, &olo, &ohi);
  for (const Slot& s : an.slots) {
    const coot_mat& L = leaves[s.leaf];
    uintptr_t llo, lhi;
    strided_range(L.data, s.off, s.rs, s.cs, an.nr, an.nc, an.esz, &llo, &lhi);
    if (olo < lhi && llo < ohi) {
      const uintptr_t vorig = (uintptr_t)L.data + (uintptr_t)(s.off * an.esz);
      const bool same = !s.trans && vorig == (uintptr_t)out->data && (an.nr <= 1 || s.rs == ors) &&
                        (an.nc <= 1 || s.cs == ocs);
      if (!same)
        return set_error(COOT_ERR_ALIAS, "out overlaps leaf %d through a %s read; only an identical read may alias",
                         s.leaf, s.trans ? "transposed" : "differently shaped or strided");
    }
  }
  return COOT_OK;
}

// ---------------------------------------------------------------------------
// kernel choice
// ---------------------------------------------------------------------------
Choice choose(const Analysis& an, const coot_mat* leaves, const coot_mat* out) {
  Choice ch;
  ch.it_rows = an.nr;
  ch.it_cols = an.nc;
  const bool out_gen = (an.gmask >> COOT_MAX_SLOTS) & 1;
  // vector accesses (16 bytes down a column) need every column start of the
  // direct reads and of a direct output 16-byte aligned; general reads and
  // writes go one element at a time and transposed reads through shared
  // memory, so neither takes part
  auto aligned = [&](bool collapsed) {
    for (const Slot& s : an.slots) {
      if (s.trans || s.gen) continue;
      const coot_mat& L = leaves[s.leaf];
      const uintptr_t org = (uintptr_t)L.data + (uintptr_t)(s.off * an.esz);
      if (org % 16) return false;
      if (!collapsed && an.nc > 1 && (s.cs * an.esz) % 16) return false;
    }
    if (out && !out_gen) {
      if ((uintptr_t)out->data % 16) return false;
      if (!collapsed && an.nc > 1 && (mat_ld(*out) * an.esz) % 16) return false;
    }
    return true;
  };
  if (an.any_trans && !(an.scan() && an.scan_direct)) {
    // a reduction along dim 1 whose transposed reads are no more than its
    // direct streams: the row walk, reading each transposed slot along the
    // thread's run of columns; else the tiles, staged through shared memory
    int ntr = 0, ndir = 0;
    for (const Slot& s : an.slots) {
      if (s.trans) ++ntr;
      else if (!s.gen) ++ndir;
    }
    if (out) ++ndir;
    const bool along1 = an.red.kind != COOT_R_NONE && !an.scan() && an.red.dim == 1 && an.n_seg() == 1;
    ch.fam = (along1 && ntr <= ndir) ? F_ROW : F_TILE;
    ch.vec_ok = aligned(false);
    return ch;
  }
  const int dim = an.red.dim;
  if (an.scan()) {
    // cumsum: warps down the columns or threads along the rows, never collapsed
    ch.fam = F_SCAN;
    ch.vec_ok = aligned(false);
    return ch;
  }
  // every kind that takes a dim: sum, mean, var, stddev, min, max, index_*, prod
  const bool along = an.red.kind != COOT_R_NONE && dim >= 0;
  if (along && dim == 0)
    ch.fam = F_COL;
  else if (along && dim == 1)
    ch.fam = F_ROW;
  else
    ch.fam = F_STR;
  // contiguity of every read and of the output: the tree is one long column
  bool contig = true;
  for (const Slot& s : an.slots)
    if (s.gen || (an.nc > 1 && s.cs != an.nr)) contig = false;
  if (out && (out_gen || (an.nc > 1 && mat_ld(*out) != an.nr))) contig = false;
  if (ch.fam == F_STR && contig) {
    ch.collapsed = true;
    ch.it_rows = an.nr * an.nc;
    ch.it_cols = (ch.it_rows > 0) ? 1 : 0;
  }
  ch.vec_ok = aligned(ch.collapsed);
  return ch;
}

// ---------------------------------------------------------------------------
// code generation
// ---------------------------------------------------------------------------
static int vmax(const Analysis& an) { return 16 / an.esz; }

Program make_program(const Analysis& an, Family fam, bool var_two_pass, bool bounds) {
  Program pg;
  const std::string S = storage_type_name(an.dtype);
  const int NS = (int)an.slots.size(), NK = (int)an.scalars.size();
  const bool OUT = an.has_out;
  const int V = vmax(an);
  std::ostringstream src, sig;
  if (an.gmask) src << "#define COOT_GM " << an.gmask << "\n";
  if (bounds) src << "#define COOT_DEBUG_BOUNDS 1\n";
  if (an.accum == 1) src << "#define COOT_ACCUM_KAHAN 1\n";
  if (an.accum == 2) src << "#define COOT_ACCUM_PLAIN 1\n";
  src << (fam == F_GEMM ? "#include \"coot_gemm.cuh\"\n" : "#include \"coot_kernels.cuh\"\n")
      << "using namespace coot;\n";
  src << "typedef " << S << " S_t;\n";
  src << "typedef " << an.type_str << " T_t;\n";
  // minb > 0: at least minb resident blocks per SM (caps registers per thread)
  auto wrap = [&](const std::string& name, int bound, const std::string& body, const char* ptype = "Params",
                  int minb = 0) {
    src << "extern \"C\" __global__ void __launch_bounds__(" << bound;
    if (minb > 0) src << ", " << minb;
    src << ") " << name << "(const __grid_constant__ " << ptype << " p) { " << body << "(p); }\n";
  };
  auto add = [&](const std::string& name, int vec, int unroll, int block) {
    KernelSpec k;
    k.name = name;
    k.vec = vec;
    k.unroll = unroll;
    k.block = block;
    pg.kernels.push_back(k);
  };
  auto red_name = [](int m) {
    switch (m) {
      case RED_NONE: return "RED_NONE";
      case RED_SUM: return "RED_SUM";
      case RED_DOT: return "RED_DOT";
      case RED_SSQ: return "RED_SSQ";
      case RED_MEAN1: return "RED_MEAN1";
      case RED_CSQ: return "RED_CSQ";
      case RED_MIN: return "RED_MIN";
      case RED_MAX: return "RED_MAX";
      case RED_IMIN: return "RED_IMIN";
      case RED_IMAX: return "RED_IMAX";
      case RED_PROD: return "RED_PROD";
    }
    return "RED_NONE";
  };
  const char* outs = OUT ? "true" : "false";
  char buf[512];
  // (vector width, unroll) variants of the column-walking families; the
  // scalar variant serves unaligned calls
  std::vector<std::pair<int, int>> vu = {{V, 1}, {V, 2}, {V, 4}, {1, 4}};
  if (fam == F_STR) {
    for (auto [v, u] : vu) {
      if (var_two_pass) {
        snprintf(buf, sizeof buf, "coot_str_p1_v%du%d", v, u);
        wrap(buf, 512, std::string("str_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) +
                            ", RED_MEAN1, " + std::to_string(v) + ", " + std::to_string(u) + ", false>");
        add(buf, v, u, 512);
        snprintf(buf, sizeof buf, "coot_str_p2_v%du%d", v, u);
        wrap(buf, 512, std::string("str_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) +
                            ", RED_CSQ, " + std::to_string(v) + ", " + std::to_string(u) + ", " + outs + ">");
        add(buf, v, u, 512);
      } else {
        snprintf(buf, sizeof buf, "coot_str_v%du%d", v, u);
        wrap(buf, 512, std::string("str_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) + ", " +
                            red_name(an.red_mode) + ", " + std::to_string(v) + ", " + std::to_string(u) + ", " + outs +
                            ">");
        add(buf, v, u, 512);
      }
    }
  } else if (fam == F_COL || fam == F_ROW) {
    const char* fn = (fam == F_COL) ? "col" : "row";
    std::vector<std::pair<int, int>> cvu = {{V, 1}, {V, 2}, {V, 4}, {1, 4}};
    // transposed reads (the row walk only): a row per thread, runs of
    // consecutive columns (the first length listed is the default)
    if (an.any_trans) {
      if (an.esz == 8)
        cvu = {{1, 8}, {1, 4}, {1, 16}};  // 64-byte runs of 8-byte values
      else
        cvu = {{1, 16}, {1, 8}, {1, 4}};
    }
    // (an empty reduction of a transposed tree may take the column family:
    // it reads nothing, so its kernels need no transposed form)
    const std::string tr = (an.any_trans && fam == F_ROW) ? ", " + std::to_string(an.trmask) : std::string();
    auto one = [&](const char* pass, const char* red, const char* o, int v, int u) {
      snprintf(buf, sizeof buf, "coot_%s%s_v%du%d", fn, pass, v, u);
      wrap(buf, 512, std::string(fn) + "_kernel<T_t, S_t, " + std::to_string(NS) + ", " + std::to_string(NK) + ", " +
                          red + ", " + std::to_string(v) + ", " + std::to_string(u) + ", " + o + tr + ">");
      add(buf, v, u, 512);
    };
    for (auto [v, u] : cvu) {
      if (var_two_pass) {
        one("_p1", "RED_MEAN1", "false", v, u);
        one("_p2", "RED_CSQ", outs, v, u);
      } else {
        one("", red_name(an.red_mode), outs, v, u);
      }
    }
  } else if (fam == F_TILE) {
    const int dim = an.red.dim;
    // vectorised variant (no dim reduction) when its staged tiles fit in
    // static shared memory: NTR x 32 x (32 V + pad) values of the compute type
    int ntr = 0;
    for (size_t s = 0; s < an.slots.size(); ++s) ntr += an.slots[s].trans ? 1 : 0;
    const int csize = (an.ct == CT_F64) ? 8 : 4;
    const int tm = 32 * V, sp = tm + 16 / csize;
    // static shared memory: staged tiles, plus the reduction scratch
    // (32 + 256 + max(TM, 32) accumulators)
    const int ab = an.acc_bytes();
    const bool tv = (ntr * 32 * sp * csize + (32 + 256 + std::max(tm, 32)) * ab + 16 <= 49152);
    // register caps: the tile kernel at 4 resident blocks (64 registers);
    // tilev at 3 (80), with 2 and 4 as tuning alternatives; tilev of 16-bit
    // storage (32-byte vectors, twice the values in flight) at 2
    auto tilev = [&](const char* name, const char* red, int minb) {
      wrap(name, 256,
           std::string("tilev_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) + ", " + red + ", " +
               std::to_string(dim) + ", " + std::to_string(an.trmask) + ", " +
               (std::string(name).find("_p1") != std::string::npos ? "false" : outs) + ", " + std::to_string(V) + ">",
           "Params", minb);
      add(name, V, 2, 256);
    };
    auto tile = [&](const char* name, const char* red, const char* o) {
      wrap(name, 256,
           std::string("tile_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) + ", " + red + ", " +
               std::to_string(dim) + ", " + std::to_string(an.trmask) + ", " + o + ">",
           "Params", 4);
      add(name, 1, 1, 256);
    };
    const int tv_minb = (an.esz == 2) ? 2 : 3;
    if (var_two_pass) {
      if (tv) {
        tilev("coot_tilev_p1", "RED_MEAN1", tv_minb);
        tilev("coot_tilev_p2", "RED_CSQ", tv_minb);
      }
      tile("coot_tile_p1", "RED_MEAN1", "false");
      tile("coot_tile_p2", "RED_CSQ", outs);
    } else {
      tile("coot_tile", red_name(an.red_mode), outs);
      if (tv) {
        tilev("coot_tilev", red_name(an.red_mode), tv_minb);
        if (an.esz != 2) {
          tilev("coot_tilev_o2", red_name(an.red_mode), 2);
          tilev("coot_tilev_o4", red_name(an.red_mode), 4);
        }
      }
    }
  } else if (fam == F_SCAN) {
    // cumsum: totals pass (_t_, used when the lines are cut into segments)
    // and scan pass per vector variant
    if (an.red.dim == 0) {
      for (int v : {V, 1}) {
        for (int pass : {1, 2}) {
          snprintf(buf, sizeof buf, pass == 1 ? "coot_scan_t_v%d" : "coot_scan_v%d", v);
          wrap(buf, 256, std::string("scan_col_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) +
                             ", " + std::to_string(v) + ", " + std::to_string(pass) + ">");
          add(buf, v, 1, 256);
        }
      }
    } else if (an.any_trans) {
      // transposed reads: the one-pass row scan only (a row per thread, the
      // transposed slots read along the thread's runs of columns)
      snprintf(buf, sizeof buf, "coot_scanp_v1u16w8");
      wrap(buf, 256,
           std::string("scanp_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) + ", 1, 16, 8, " +
               std::to_string(an.trmask) + ">",
           "Params", 2);
      add(buf, 1, 16, 256);
    } else {
      std::vector<std::pair<int, int>> svu = {{V, 2}, {V, 4}, {1, 4}};
      for (auto [v, u] : svu) {
        for (int pass : {1, 2}) {
          snprintf(buf, sizeof buf, pass == 1 ? "coot_scan_t_v%du%d" : "coot_scan_v%du%d", v, u);
          wrap(buf, 256, std::string("scan_row_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) +
                             ", " + std::to_string(v) + ", " + std::to_string(u) + ", " + std::to_string(pass) + ">");
          add(buf, v, u, 256);
        }
      }
      // one pass over bands of 32 v rows, panels of nw warps x uc columns
      struct Pv { int v, uc, nw, minb; };
      // (V = 1: two resident blocks per SM, as the bands of a tall matrix
      // outnumber the SMs by less than two)
      std::vector<Pv> pvu = {{1, 16, 8, 2}};
      if (V >= 2) pvu.push_back({2, 8, 8, 0});
      for (const Pv& q : pvu) {
        snprintf(buf, sizeof buf, "coot_scanp_v%du%dw%d", q.v, q.uc, q.nw);
        wrap(buf, 32 * q.nw,
             std::string("scanp_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) + ", " +
                 std::to_string(q.v) + ", " + std::to_string(q.uc) + ", " + std::to_string(q.nw) + ">",
             "Params", q.minb);
        add(buf, q.v, q.uc, 32 * q.nw);
      }
    }
  } else if (fam == F_GEMM && an.esz != 2) {
    // FP32 / FP64 operands: the CUDA-core kernel, 256 threads, 2 blocks per SM
    wrap("coot_gemm_simt", 256,
         std::string("gemm_simt_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) + ", " +
             std::to_string(an.gemm_ps) + ", " + (an.gemm_ka ? "true" : "false") + ", " +
             (an.gemm_kb ? "true" : "false") + ">",
         "GemmParams", 2);
    add("coot_gemm_simt", 1, 1, 256);
  } else if (fam == F_GEMM) {
    // 256 threads, at least 2 blocks per SM (128 registers)
    wrap("coot_gemm", 256,
         std::string("gemm_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) + ", " +
             std::to_string(an.gemm_ps) + ", " + (an.gemm_ka ? "true" : "false") + ", " +
             (an.gemm_kb ? "true" : "false") + ">",
         "GemmParams", 2);
    add("coot_gemm", 1, 1, 256);
    // persistent tcgen05 kernel: TMA loads, accumulator in tensor memory, one CTA per SM
    wrap("coot_gemm_tc", coot::GEMM_TC_THREADS,
         std::string("gemm_tc_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) + ", " +
             std::to_string(an.gemm_ps) + ", " + (an.gemm_ka ? "true" : "false") + ", " +
             (an.gemm_kb ? "true" : "false") + ">",
         "GemmParams", 1);
    add("coot_gemm_tc", 1, 1, coot::GEMM_TC_THREADS);
  } else if (fam == F_ADJ) {
    std::vector<std::pair<int, int>> avu = {{V, 1}, {V, 2}, {1, 4}};
    for (auto [v, u] : avu) {
      snprintf(buf, sizeof buf, "coot_adj_v%du%d", v, u);
      wrap(buf, 512, std::string("adj_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) + ", " +
                          std::to_string(v) + ", " + std::to_string(u) + ">");
      add(buf, v, u, 512);
    }
  } else if (fam == F_BATCH) {
    const bool red = an.red_mode != RED_NONE;
    wrap("coot_batch", 256,
         std::string("batch_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) + ", " +
             std::to_string(an.trmask) + ", " + (red ? "true" : "false") + ">",
         "BatchParams");
    add("coot_batch", 1, 1, 256);
    // the flat walk over work items (the default)
    wrap("coot_batchf", coot::BATCHF_THREADS,
         std::string("batchf_kernel<T_t, S_t, ") + std::to_string(NS) + ", " + std::to_string(NK) + ", " +
             std::to_string(an.trmask) + ", " + (red ? "true" : "false") + ", " + std::to_string(an.batch_be) + ">",
         "BatchParams", an.batch_minb);
    add("coot_batchf", 1, 1, coot::BATCHF_THREADS);
  }
  sig << "cootgb1|" << family_name(fam) << "|" << S << "|ns" << NS << "|nk" << NK << "|red" << an.red_mode << "|dim"
      << an.red.dim << "|out" << OUT << "|tr" << an.trmask << "|gm" << an.gmask << "|var" << var_two_pass
      << (fam == F_GEMM ? "|ps" + std::to_string(an.gemm_ps) + (an.gemm_ka ? "ka" : "ma") + (an.gemm_kb ? "kb" : "nb")
                        : std::string())
      << (an.accum == 1 ? "|kahan" : (an.accum == 2 ? "|plain" : ""))
      << (fam == F_BATCH ? "|be" + std::to_string(an.batch_be) + "b" + std::to_string(an.batch_minb) : std::string())
      << (bounds ? "|bounds" : "")
      << "|" << an.type_str;
  pg.signature = sig.str();
  pg.source = src.str();
  return pg;
}

}  // namespace cg
