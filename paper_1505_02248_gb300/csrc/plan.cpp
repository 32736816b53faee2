// Host-side planning: descriptor validation, owner tiles D_i and windows M_i
// (Sec. 3, Fig. 3), and grouping of windows with identical local operators.
#include <cmath>
#include <map>
#include <tuple>

#include "lem_internal.h"

namespace lem {

lem_status validate(const lem_problem_desc* d) {
  if (!d) return fail(LEM_EINVAL, "descriptor is NULL");
  if (d->ndim != 1 && d->ndim != 2) return fail(LEM_EINVAL, "ndim must be 1 or 2");
  for (int a = 0; a < d->ndim; ++a) {
    if (d->n[a] < 1 || d->n[a] > (int64_t(1) << 24)) return fail(LEM_EINVAL, "n out of range [1, 2^24]");
    if (d->bc[a] != LEM_BC_DIRICHLET0 && d->bc[a] != LEM_BC_PERIODIC) return fail(LEM_EINVAL, "bad bc");
    if (d->tile[a] < 1) return fail(LEM_EINVAL, "tile must be >= 1");
    if (d->overlap[a] < 0) return fail(LEM_EINVAL, "overlap must be >= 0");
  }
  int64_t npts = d->ndim == 1 ? d->n[0] : d->n[0] * d->n[1];
  if (npts > (int64_t(1) << 31)) return fail(LEM_EINVAL, "mesh larger than 2^31 nodes");
  if (!(d->dt > 0.0) || !std::isfinite(d->dt)) return fail(LEM_EINVAL, "dt must be finite and > 0");
  if (d->coef_stride != 0 && d->coef_stride != 1) return fail(LEM_EINVAL, "coef_stride must be 0 or 1");
  int ncoef = d->ndim == 1 ? 3 : 5;
  for (int k = 0; k < ncoef; ++k)
    if (!d->coef[k]) return fail(LEM_EINVAL, "missing stencil coefficient pointer");
  if (d->mode != LEM_MODE_PHI && d->mode != LEM_MODE_EXP) return fail(LEM_EINVAL, "bad mode");
  if (d->prec != LEM_PREC_FP64 && d->prec != LEM_PREC_SPLIT && d->prec != LEM_PREC_SPLIT_FAST)
    return fail(LEM_EINVAL, "bad prec");
  if (d->reaction < 0 || d->reaction > 2) return fail(LEM_EINVAL, "reaction must be 0, 1 or 2");
  if (d->reaction == 2 && !(d->porous_m > 1.0 && std::isfinite(d->porous_m)))
    return fail(LEM_EINVAL, "porous_m must be finite and > 1");
  if (d->reaction == 2 && d->scheme != LEM_SCHEME_EULER)
    return fail(LEM_EINVAL, "the porous-medium problem runs the exponential Euler scheme");
  if (d->reaction && d->mode != LEM_MODE_PHI) return fail(LEM_EINVAL, "the reaction needs LEM_MODE_PHI");
  if (d->refresh < 0) return fail(LEM_EINVAL, "refresh must be >= 0");
  if (d->scheme != LEM_SCHEME_EULER && d->scheme != LEM_SCHEME_RB3) return fail(LEM_EINVAL, "bad scheme");
  if (d->scheme == LEM_SCHEME_RB3 && d->mode != LEM_MODE_PHI)
    return fail(LEM_EINVAL, "the third-order Rosenbrock scheme needs LEM_MODE_PHI");
  if (d->complex_values != 0 && d->complex_values != 1) return fail(LEM_EINVAL, "complex_values must be 0 or 1");
  if (d->complex_values && (d->reaction || d->scheme != LEM_SCHEME_EULER))
    return fail(LEM_EINVAL, "complex problems are linear, with the exponential Euler scheme");
  return LEM_OK;
}

namespace {
struct AxisTile {
  int32_t org, wext, iofs, iext, t0, whole;
};

std::vector<AxisTile> axis_tiles(int64_t n, int tile, int H, bool periodic) {
  std::vector<AxisTile> out;
  for (int64_t t0 = 0; t0 < n; t0 += tile) {
    int64_t t1 = std::min<int64_t>(t0 + tile, n);  // the last tile may be ragged
    AxisTile a{};
    a.t0 = int32_t(t0);
    a.iext = int32_t(t1 - t0);
    if (periodic) {
      if ((t1 - t0) + 2 * int64_t(H) >= n) {  // window reaches around: the whole axis
        a.org = 0; a.wext = int32_t(n); a.iofs = int32_t(t0); a.whole = 1;
      } else {
        a.org = int32_t(t0 - H); a.wext = int32_t((t1 - t0) + 2 * H); a.iofs = H; a.whole = 0;
      }
    } else {  // clipped at the walls: no node exists beyond the mesh
      int64_t lo = std::max<int64_t>(0, t0 - H), hi = std::min<int64_t>(n, t1 + H);
      a.org = int32_t(lo); a.wext = int32_t(hi - lo); a.iofs = int32_t(t0 - lo); a.whole = 0;
    }
    out.push_back(a);
  }
  return out;
}
}  // namespace

lem_status make_plan(lem_ctx* ctx) {
  const lem_problem_desc& d = ctx->desc;
  std::vector<AxisTile> ay, ax;
  if (d.ndim == 1) {
    ay.push_back(AxisTile{0, 1, 0, 1, 0, 0});
    ax = axis_tiles(d.n[0], d.tile[0], d.overlap[0], d.bc[0] == LEM_BC_PERIODIC);
  } else {
    ay = axis_tiles(d.n[0], d.tile[0], d.overlap[0], d.bc[0] == LEM_BC_PERIODIC);
    ax = axis_tiles(d.n[1], d.tile[1], d.overlap[1], d.bc[1] == LEM_BC_PERIODIC);
  }
  const bool shared = d.coef_stride == 0 && !d.reaction;  // identical operators can be shared
  std::map<std::tuple<int, int, int, int, int, int, int, int>, int32_t> keymap;
  ctx->tiles.clear();
  ctx->classes.clear();
  ctx->n_loc = ctx->n_int = 0;
  for (const AxisTile& y : ay) {
    for (const AxisTile& x : ax) {
      TileDesc t{};
      t.org[0] = y.org; t.org[1] = x.org;
      t.wext[0] = y.wext; t.wext[1] = x.wext;
      t.iofs[0] = y.iofs; t.iofs[1] = x.iofs;
      t.iext[0] = y.iext; t.iext[1] = x.iext;
      t.t0[0] = y.t0; t.t0[1] = x.t0;
      int32_t cls;
      auto key = std::make_tuple(y.wext, x.wext, y.iofs, x.iofs, y.iext, x.iext, y.whole, x.whole);
      auto it = shared ? keymap.find(key) : keymap.end();
      if (it == keymap.end()) {
        cls = int32_t(ctx->classes.size());
        ClassDesc c{};
        c.rep_tile = int32_t(ctx->tiles.size());
        c.wext[0] = y.wext; c.wext[1] = x.wext;
        c.iext[0] = y.iext; c.iext[1] = x.iext;
        c.iofs[0] = y.iofs; c.iofs[1] = x.iofs;
        c.whole[0] = y.whole; c.whole[1] = x.whole;
        ctx->classes.push_back(c);
        if (shared) keymap[key] = cls;
      } else {
        cls = it->second;
      }
      t.cls = cls;
      ctx->classes[cls].ntiles++;
      ctx->n_loc = std::max<int64_t>(ctx->n_loc, int64_t(t.wext[0]) * t.wext[1]);
      ctx->n_int = std::max<int64_t>(ctx->n_int, int64_t(t.iext[0]) * t.iext[1]);
      ctx->tiles.push_back(t);
    }
  }
  if (ctx->n_loc > 16384) return fail(LEM_EINVAL, "window larger than 16384 nodes (dense local matrices)");
  // tiles grouped by class (stable), for grouped application
  const size_t nc = ctx->classes.size();
  ctx->class_offset.assign(nc + 1, 0);
  for (const TileDesc& t : ctx->tiles) ctx->class_offset[t.cls + 1]++;
  for (size_t c = 0; c < nc; ++c) ctx->class_offset[c + 1] += ctx->class_offset[c];
  ctx->class_order.assign(ctx->tiles.size(), 0);
  std::vector<int32_t> fill(ctx->class_offset.begin(), ctx->class_offset.end() - 1);
  for (size_t i = 0; i < ctx->tiles.size(); ++i) ctx->class_order[fill[ctx->tiles[i].cls]++] = int32_t(i);
  ctx->squarings.assign(nc, -1);
  return LEM_OK;
}

}  // namespace lem
