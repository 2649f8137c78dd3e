// Supernodal nested dissection of a quasi-2D box (§2.1 and its separator-tree figure).
//
// Rule (the paper gives it only as a figure): a box [x0,x1) x [y0,y1) x all planes is a leaf
// when wx*wy*depth <= leaf; otherwise the longer side is cut (ties cut x) by the whole-depth
// plane at mid = x0 + wx/2 (resp. y0 + wy/2); the two remaining boxes are the children (empty
// ones dropped).  Postorder numbering: low child subtree, high child subtree, separator.
// Inside a supernode nodes run x fastest, then y, then z.  struct(S) of a supernode whose
// subtree covers box B is the set of in-domain nodes adjacent to B, i.e. the four side strips
// of B over every plane (the shallow direction is never cut), sorted by elimination index.
#include <algorithm>
#include <stdexcept>

#include "psp_internal.h"

namespace psp {

namespace {

struct Builder {
  Shape& sh;
  std::vector<int32_t> box;       // 4 per supernode: x0 x1 y0 y1 of its subtree region
  std::vector<std::vector<int32_t>> nodes;
  std::vector<std::vector<int32_t>> kids;

  explicit Builder(Shape& s) : sh(s) {}

  void add_nodes(std::vector<int32_t>& out, int x0, int x1, int y0, int y1) {
    for (int z = 0; z < sh.nz; ++z)
      for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) out.push_back(x + sh.nx * (y + sh.ny * z));
  }

  int rec(int x0, int x1, int y0, int y1) {
    int wx = x1 - x0, wy = y1 - y0;
    if (wx <= 0 || wy <= 0) return -1;
    std::vector<int32_t> mine;
    std::vector<int32_t> ch;
    if ((int64_t)wx * wy * sh.nz <= sh.leaf) {
      add_nodes(mine, x0, x1, y0, y1);
    } else if (wx >= wy) {
      int mid = x0 + wx / 2;
      int a = rec(x0, mid, y0, y1);
      int b = rec(mid + 1, x1, y0, y1);
      if (a >= 0) ch.push_back(a);
      if (b >= 0) ch.push_back(b);
      add_nodes(mine, mid, mid + 1, y0, y1);
    } else {
      int mid = y0 + wy / 2;
      int a = rec(x0, x1, y0, mid);
      int b = rec(x0, x1, mid + 1, y1);
      if (a >= 0) ch.push_back(a);
      if (b >= 0) ch.push_back(b);
      add_nodes(mine, x0, x1, mid, mid + 1);
    }
    nodes.push_back(std::move(mine));
    kids.push_back(std::move(ch));
    box.insert(box.end(), {x0, x1, y0, y1});
    return (int)nodes.size() - 1;
  }
};

}  // namespace

void build_shape(Shape& sh, int nx, int ny, int nz, int leaf) {
  sh.nx = nx;
  sh.ny = ny;
  sh.nz = nz;
  sh.leaf = leaf;
  Builder b(sh);
  b.rec(0, nx, 0, ny);
  const int nsn = (int)b.nodes.size();
  sh.nsn = nsn;
  const int64_t N = (int64_t)nx * ny * nz;

  sh.first.assign(nsn + 1, 0);
  sh.s.assign(nsn, 0);
  sh.order.clear();
  sh.order.reserve(N);
  for (int f = 0; f < nsn; ++f) {
    sh.first[f] = (int32_t)sh.order.size();
    sh.s[f] = (int32_t)b.nodes[f].size();
    sh.order.insert(sh.order.end(), b.nodes[f].begin(), b.nodes[f].end());
  }
  sh.first[nsn] = (int32_t)sh.order.size();
  if ((int64_t)sh.order.size() != N) throw std::runtime_error("nested dissection lost nodes");
  sh.elim.assign(N, -1);
  for (int64_t e = 0; e < N; ++e) sh.elim[sh.order[e]] = (int32_t)e;

  sh.parent.assign(nsn, -1);
  sh.child_ptr.assign(nsn + 1, 0);
  sh.child_idx.clear();
  for (int f = 0; f < nsn; ++f) {
    sh.child_ptr[f] = (int32_t)sh.child_idx.size();
    for (int c : b.kids[f]) {
      sh.child_idx.push_back(c);
      sh.parent[c] = f;
    }
  }
  sh.child_ptr[nsn] = (int32_t)sh.child_idx.size();

  // struct(S): side strips of the subtree box, sorted by elimination index
  sh.struct_ptr.assign(nsn + 1, 0);
  sh.struct_elim.clear();
  sh.u.assign(nsn, 0);
  std::vector<int32_t> tmp;
  for (int f = 0; f < nsn; ++f) {
    int x0 = b.box[4 * f], x1 = b.box[4 * f + 1], y0 = b.box[4 * f + 2], y1 = b.box[4 * f + 3];
    tmp.clear();
    for (int z = 0; z < nz; ++z) {
      for (int y = y0; y < y1; ++y) {
        if (x0 > 0) tmp.push_back(sh.elim[(x0 - 1) + nx * (y + ny * z)]);
        if (x1 < nx) tmp.push_back(sh.elim[x1 + nx * (y + ny * z)]);
      }
      for (int x = x0; x < x1; ++x) {
        if (y0 > 0) tmp.push_back(sh.elim[x + nx * ((y0 - 1) + ny * z)]);
        if (y1 < ny) tmp.push_back(sh.elim[x + nx * (y1 + ny * z)]);
      }
    }
    std::sort(tmp.begin(), tmp.end());
    sh.struct_ptr[f] = (int64_t)sh.struct_elim.size();
    sh.u[f] = (int32_t)tmp.size();
    sh.struct_elim.insert(sh.struct_elim.end(), tmp.begin(), tmp.end());
  }
  sh.struct_ptr[nsn] = (int64_t)sh.struct_elim.size();

  // relative positions of each struct entry within the parent's front rows (S_p, struct(S_p))
  sh.rel.assign(sh.struct_elim.size(), -1);
  for (int f = 0; f < nsn; ++f) {
    int p = sh.parent[f];
    if (p < 0) {
      if (sh.u[f] != 0) throw std::runtime_error("root with non-empty struct");
      continue;
    }
    const int32_t* ps = sh.struct_elim.data() + sh.struct_ptr[p];
    for (int64_t a = sh.struct_ptr[f]; a < sh.struct_ptr[f + 1]; ++a) {
      int32_t e = sh.struct_elim[a];
      int32_t pos;
      if (e >= sh.first[p] && e < sh.first[p] + sh.s[p]) {
        pos = e - sh.first[p];
      } else {
        const int32_t* it = std::lower_bound(ps, ps + sh.u[p], e);
        if (it == ps + sh.u[p] || *it != e) throw std::runtime_error("struct not nested in parent front");
        pos = sh.s[p] + (int32_t)(it - ps);
      }
      sh.rel[a] = pos;
    }
  }

  // heights and level lists
  sh.height.assign(nsn, 0);
  int hmax = 0;
  for (int f = 0; f < nsn; ++f) {
    int h = 0;
    for (int32_t c = sh.child_ptr[f]; c < sh.child_ptr[f + 1]; ++c) h = std::max(h, sh.height[sh.child_idx[c]] + 1);
    sh.height[f] = h;
    hmax = std::max(hmax, h);
  }
  sh.nlevels = hmax + 1;
  sh.level_sns.assign(sh.nlevels, {});
  for (int f = 0; f < nsn; ++f) sh.level_sns[sh.height[f]].push_back(f);
  // depths (root 0, child = parent + 1; postorder puts every parent after its children)
  sh.depth.assign(nsn, 0);
  int dmax = 0;
  for (int f = nsn - 1; f >= 0; --f) {
    if (sh.parent[f] >= 0) sh.depth[f] = sh.depth[sh.parent[f]] + 1;
    dmax = std::max(dmax, (int)sh.depth[f]);
  }
  sh.ndepths = dmax + 1;

  // per-panel layouts: G blocks (padded to 16 elements) and update vectors
  sh.g_off.assign(nsn, 0);
  sh.upd_off.assign(nsn, 0);
  int64_t go = 0, uo = 0;
  for (int f = 0; f < nsn; ++f) {
    sh.g_off[f] = go;
    go += ((int64_t)(sh.s[f] + sh.u[f]) * sh.s[f] + 15) / 16 * 16;
    sh.upd_off[f] = uo;
    uo += sh.u[f];
  }
  sh.g_total = go;
  sh.upd_total = std::max<int64_t>(uo, 1);

  // pull map of the solve: children's update entries landing on each front row position
  sh.pull_ptr.assign(nsn + 1, 0);
  int64_t pp = 0;
  for (int f = 0; f < nsn; ++f) {
    sh.pull_ptr[f] = pp;
    pp += sh.s[f] + sh.u[f];
  }
  sh.pull_ptr[nsn] = pp;
  sh.pull.assign(2 * pp, -1);
  for (int f = 0; f < nsn; ++f) {
    int p = sh.parent[f];
    if (p < 0) continue;
    for (int64_t a = sh.struct_ptr[f]; a < sh.struct_ptr[f + 1]; ++a) {
      int64_t slot = 2 * (sh.pull_ptr[p] + sh.rel[a]);
      int32_t val = (int32_t)(sh.upd_off[f] + (a - sh.struct_ptr[f]));
      if (sh.pull[slot] < 0) sh.pull[slot] = val;
      else if (sh.pull[slot + 1] < 0) sh.pull[slot + 1] = val;
      else throw std::runtime_error("more than two children update one position");
    }
  }
}

}  // namespace psp
