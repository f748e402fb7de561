// Host-side scene preprocessing (native): validation, rest data, surface
// extraction, SELL-32 pattern with degree-sorted rows and assembly maps,
// contact-vertex / object tables.  Pure C++; no CUDA calls.
//
// Each env is first built in env-local indices (EnvLocal); identical
// consecutive descriptors reuse the previous EnvLocal, then everything is
// appended to the flat Pack with global offsets.
#include "scene.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <numeric>

namespace ipc {

struct BodyProps {
  double vol, mass, com[3], S[9];
};

// Mass properties of a closed outward triangle surface by the divergence
// theorem applied to tetrahedra fanned from the first vertex q0: each
// triangle (a, b, c) contributes the signed tet (q0, a, b, c).
bool body_props(const double* X, int nv, const int* T, int nt, double rho, BodyProps& out) {
  if (nv < 4 || nt < 4) return false;
  const double* o = X;
  double vol = 0, m1[3] = {0, 0, 0}, m2[9] = {0};
  for (int t = 0; t < nt; ++t) {
    double q[3][3];
    for (int k = 0; k < 3; ++k) {
      int v = T[3 * t + k];
      if (v < 0 || v >= nv) return false;
      for (int c = 0; c < 3; ++c) q[k][c] = X[3 * v + c] - o[c];
    }
    double cx = q[0][1] * q[1][2] - q[0][2] * q[1][1];
    double cy = q[0][2] * q[1][0] - q[0][0] * q[1][2];
    double cz = q[0][0] * q[1][1] - q[0][1] * q[1][0];
    double V = (cx * q[2][0] + cy * q[2][1] + cz * q[2][2]) / 6.0;
    vol += V;
    double s[3];
    for (int c = 0; c < 3; ++c) {
      s[c] = q[0][c] + q[1][c] + q[2][c];
      m1[c] += V * s[c] / 4.0;
    }
    // int x x^T over the tet (origin corner is 0): V/20 (sum q q^T + s s^T)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = s[i] * s[j];
        for (int k = 0; k < 3; ++k) acc += q[k][i] * q[k][j];
        m2[3 * i + j] += V * acc / 20.0;
      }
  }
  if (!(vol > 0)) return false;
  double c[3] = {m1[0] / vol, m1[1] / vol, m1[2] / vol};
  out.vol = vol;
  out.mass = rho * vol;
  for (int k = 0; k < 3; ++k) out.com[k] = o[k] + c[k];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) out.S[3 * i + j] = rho * (m2[3 * i + j] - vol * c[i] * c[j]);
  return true;
}

double det3d(const double* a) {
  return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
         a[2] * (a[3] * a[7] - a[4] * a[6]);
}

void inv3d(const double* a, double* r) {
  double d = det3d(a);
  r[0] = (a[4] * a[8] - a[5] * a[7]) / d;
  r[1] = (a[2] * a[7] - a[1] * a[8]) / d;
  r[2] = (a[1] * a[5] - a[2] * a[4]) / d;
  r[3] = (a[5] * a[6] - a[3] * a[8]) / d;
  r[4] = (a[0] * a[8] - a[2] * a[6]) / d;
  r[5] = (a[2] * a[3] - a[0] * a[5]) / d;
  r[6] = (a[3] * a[7] - a[4] * a[6]) / d;
  r[7] = (a[1] * a[6] - a[0] * a[7]) / d;
  r[8] = (a[0] * a[4] - a[1] * a[3]) / d;
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// One env in env-local indices.
struct EnvLocal {
  EnvInfo info;
  double mu = 0, lam = 0;
  // rows
  std::vector<double> row_mass, row_xbar, rest_x;
  std::vector<uint8_t> row_kind;
  std::vector<int> row_body;           // local body or -1
  std::vector<int> vt_ptr, vt_src;     // src: local tet*4 + a
  // tets
  std::vector<int> tets;               // local rows
  std::vector<double> Dm_inv, vol;
  // SELL
  std::vector<int> chunk_slots;
  std::vector<long long> chunk_ptr;    // local block offsets
  std::vector<int> sell_col;           // local rows
  std::vector<int> asm_ptr, asm_src;   // src: local tet*16 + a*4 + b
  long long n_blocks = 0;
  // bodies
  std::vector<BodyProps> bp;
  std::vector<int> body_cv0, body_driven;
  std::vector<double> body_kappa;
  // contact
  std::vector<int> cv_row, cv_body, cv_obj, cv_uid;   // local
  std::vector<double> cv_xbar, cv_area;
  std::vector<uint8_t> cv_fixed;
  std::vector<int> tri, tri_obj, edge, edge_obj;
  std::vector<double> edge_area, edge_len2;
  std::vector<int> obj_cvb, obj_cve, obj_tb, obj_te, obj_eb, obj_ee;
  std::vector<unsigned long long> obj_ex;
  std::vector<int> coated_row;
  // broad-phase hierarchy: per kind (0 points, 1 triangles, 2 edges) the
  // object's primitives in Morton order of their rest centroids (local ids)
  std::vector<int> bv_ord[3];
};

namespace {

// 21-bit spread for a 63-bit Morton key
static unsigned long long morton_spread(unsigned long long v) {
  v &= 0x1fffffull;
  v = (v | v << 32) & 0x1f00000000ffffull;
  v = (v | v << 16) & 0x1f0000ff0000ffull;
  v = (v | v << 8) & 0x100f00f00f00f00full;
  v = (v | v << 4) & 0x10c30c30c30c30c3ull;
  v = (v | v << 2) & 0x1249249249249249ull;
  return v;
}

// Primitives [b, e) of one object, given their rest centroids (3 per
// primitive, indexed from b), in Morton order of the centroids within the
// object's box; ties keep index order.  Appended to ord.
static void morton_order(int b, int e, const std::vector<double>& cen, std::vector<int>& ord) {
  if (e <= b) return;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = b; i < e; ++i)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], cen[3 * (i - b) + c]);
      hi[c] = std::max(hi[c], cen[3 * (i - b) + c]);
    }
  std::vector<std::pair<unsigned long long, int>> key;
  key.reserve(e - b);
  for (int i = b; i < e; ++i) {
    unsigned long long k = 0;
    for (int c = 0; c < 3; ++c) {
      const double ext = hi[c] - lo[c];
      const double u = ext > 0 ? (cen[3 * (i - b) + c] - lo[c]) / ext : 0.0;
      const unsigned long long q = (unsigned long long)std::min(2097151.0, std::max(0.0, u * 2097151.0));
      k |= morton_spread(q) << c;
    }
    key.push_back({k, i});
  }
  std::stable_sort(key.begin(), key.end(), [](const std::pair<unsigned long long, int>& x,
                                              const std::pair<unsigned long long, int>& y) { return x.first < y.first; });
  for (auto& kv : key) ord.push_back(kv.second);
}

bool build_local(const ipc_scene_desc& s, int e, const ipc_params& prm, EnvLocal& L, std::string& err) {
  char buf[256];
  const int N = s.n_verts, T = s.n_tets, nb = s.n_bodies;
  if (N < 4 || T < 1 || !s.rest_x || !s.tets || nb < 0 ||
      (nb > 0 && (!s.body_nv || !s.body_rest_x || !s.body_nt || !s.body_tris || !s.body_rho ||
                  !s.body_kappa_s || !s.body_driven))) {
    snprintf(buf, sizeof buf, "env %d: missing or empty scene arrays", e);
    err = buf;
    return false;
  }
  if (!(s.E > 0) || !(s.nu > -1 && s.nu < 0.5) || !(s.rho > 0)) {
    snprintf(buf, sizeof buf, "env %d: invalid material (E, nu, rho)", e);
    err = buf;
    return false;
  }
  EnvInfo& ev = L.info;
  ev.n_verts = N; ev.n_tets = T; ev.n_bodies = nb;
  std::vector<int> pad(N, 0);
  if (s.pad_id)
    for (int i = 0; i < N; ++i) {
      pad[i] = s.pad_id[i];
      if (pad[i] < 0 || pad[i] >= MAX_OBJECTS_PER_ENV) { err = "pad_id out of range"; return false; }
    }
  const int n_pads = 1 + *std::max_element(pad.begin(), pad.end());
  ev.n_pads = n_pads;
  if (n_pads + nb > MAX_OBJECTS_PER_ENV) { err = "too many contact objects in one env (max 64)"; return false; }
  std::vector<int> attach(N, -1);
  if (s.attach_body)
    for (int i = 0; i < N; ++i) {
      attach[i] = s.attach_body[i];
      if (attach[i] < -1 || attach[i] >= nb) { err = "attach_body out of range"; return false; }
    }
  auto pinned = [&](int u) { return s.pinned && s.pinned[u]; };
  // ---------------- adjacency (CSR of unique neighbours, user ids)
  for (long long k = 0; k < 4LL * T; ++k)
    if (s.tets[k] < 0 || s.tets[k] >= N) {
      snprintf(buf, sizeof buf, "env %d tet %lld: vertex out of range", e, k / 4);
      err = buf;
      return false;
    }
  std::vector<long long> pairs;
  pairs.reserve(12 * (size_t)T);
  for (int t = 0; t < T; ++t)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        if (a != b) pairs.push_back((long long)s.tets[4 * t + a] * N + s.tets[4 * t + b]);
  std::sort(pairs.begin(), pairs.end());
  pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
  std::vector<int> deg(N, 0);
  for (long long p : pairs) deg[p / N]++;
  // row order: degree descending, ties by user id
  ev.perm.resize(N);
  std::iota(ev.perm.begin(), ev.perm.end(), 0);
  std::stable_sort(ev.perm.begin(), ev.perm.end(), [&](int a, int b) { return deg[a] > deg[b]; });
  ev.inv_perm.assign(N, 0);
  for (int r = 0; r < N; ++r) ev.inv_perm[ev.perm[r]] = r;
  const int gel_rows = round_up(N, 32);
  const int body_rows = nb > 0 ? round_up(4 * nb, 32) : 0;
  const int R = round_up(gel_rows + body_rows, 128);
  ev.gel_rows = gel_rows;
  ev.n_rows = R;
  // columns per row in local rows: self first, then neighbours ascending
  std::vector<int> cptr(N + 1, 0);
  for (int r = 0; r < N; ++r) cptr[r + 1] = cptr[r] + 1 + deg[ev.perm[r]];
  std::vector<int> cidx(cptr[N]);
  {
    std::vector<int> fill(N, 1);
    for (int r = 0; r < N; ++r) cidx[cptr[r]] = r;
    for (long long p : pairs) {
      int r = ev.inv_perm[p / N], c = ev.inv_perm[p % N];
      cidx[cptr[r] + fill[r]++] = c;
    }
    for (int r = 0; r < N; ++r) std::sort(cidx.begin() + cptr[r] + 1, cidx.begin() + cptr[r + 1]);
  }
  // ---------------- material, tets, masses
  L.mu = s.E / (2.0 * (1.0 + s.nu));
  L.lam = s.E * s.nu / ((1.0 + s.nu) * (1.0 - 2.0 * s.nu));
  std::vector<double> mass(N, 0.0);
  L.tets.resize(4 * (size_t)T);
  L.Dm_inv.resize(9 * (size_t)T);
  L.vol.resize(T);
  for (int t = 0; t < T; ++t) {
    const int* q = s.tets + 4 * t;
    double Dm[9];
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) Dm[3 * i + a] = s.rest_x[3 * q[a + 1] + i] - s.rest_x[3 * q[0] + i];
    double d = det3d(Dm);
    if (!(d > 0)) {
      snprintf(buf, sizeof buf, "env %d tet %d: non-positive rest volume", e, t);
      err = buf;
      return false;
    }
    inv3d(Dm, &L.Dm_inv[9 * (size_t)t]);
    double vol = d / 6.0;
    L.vol[t] = vol;
    for (int a = 0; a < 4; ++a) {
      mass[q[a]] += s.rho * vol / 4.0;
      L.tets[4 * (size_t)t + a] = ev.inv_perm[q[a]];
    }
  }
  // ---------------- bodies
  L.bp.resize(nb);
  std::vector<int> bvoff(nb + 1, 0), btoff(nb + 1, 0);
  for (int b = 0; b < nb; ++b) {
    bvoff[b + 1] = bvoff[b] + s.body_nv[b];
    btoff[b + 1] = btoff[b] + s.body_nt[b];
  }
  for (int b = 0; b < nb; ++b) {
    if (!(s.body_rho[b] > 0) || !body_props(s.body_rest_x + 3 * bvoff[b], s.body_nv[b], s.body_tris + 3 * btoff[b],
                                            s.body_nt[b], s.body_rho[b], L.bp[b])) {
      snprintf(buf, sizeof buf, "env %d body %d: surface not closed/outward or bad density", e, b);
      err = buf;
      return false;
    }
    ev.body_com.insert(ev.body_com.end(), L.bp[b].com, L.bp[b].com + 3);
    ev.body_nv.push_back(s.body_nv[b]);
    L.body_driven.push_back(s.body_driven[b] ? 1 : 0);
    L.body_kappa.push_back(s.body_kappa_s[b]);
  }
  // ---------------- rows
  for (int r = 0; r < R; ++r) {
    double m = 0, xb[3] = {0, 0, 0}, x0[3] = {0, 0, 0};
    uint8_t kind = ROW_PAD;
    int body = -1;
    if (r < N) {
      int u = ev.perm[r];
      m = mass[u];
      for (int c = 0; c < 3; ++c) x0[c] = s.rest_x[3 * u + c];
      if (pinned(u)) kind = ROW_PINNED;
      else if (attach[u] >= 0) {
        kind = ROW_ATTACHED;
        body = attach[u];
        for (int c = 0; c < 3; ++c) xb[c] = x0[c] - L.bp[attach[u]].com[c];
      } else kind = ROW_FREE;
    } else if (r >= gel_rows && r < gel_rows + 4 * nb) {
      int b = (r - gel_rows) / 4, k = (r - gel_rows) % 4;
      kind = s.body_driven[b] ? ROW_BODY_DRIVEN : ROW_BODY;
      body = b;
      if (k == 0) for (int c = 0; c < 3; ++c) x0[c] = L.bp[b].com[c];
      else x0[k - 1] = 1.0;  // column k-1 of the identity
    }
    L.row_mass.push_back(m);
    L.row_kind.push_back(kind);
    L.row_body.push_back(body);
    L.row_xbar.insert(L.row_xbar.end(), xb, xb + 3);
    L.rest_x.insert(L.rest_x.end(), x0, x0 + 3);
  }
  // gradient gather (local tet*4 + a) per row, by counting sort
  {
    L.vt_ptr.assign(R + 1, 0);
    for (int k = 0; k < 4 * T; ++k) L.vt_ptr[L.tets[k] + 1]++;
    for (int r = 0; r < R; ++r) L.vt_ptr[r + 1] += L.vt_ptr[r];
    L.vt_src.resize(4 * (size_t)T);
    std::vector<int> fill(L.vt_ptr.begin(), L.vt_ptr.end() - 1);
    for (int k = 0; k < 4 * T; ++k) L.vt_src[fill[L.tets[k]]++] = k;
  }
  // ---------------- SELL-32
  {
    const int n_chunks = R / 32;
    L.chunk_slots.resize(n_chunks);
    L.chunk_ptr.resize(n_chunks);
    long long nblk = 0;
    for (int ch = 0; ch < n_chunks; ++ch) {
      int slots = 1;
      for (int l = 0; l < 32; ++l) {
        int r = ch * 32 + l;
        if (r < N) slots = std::max(slots, cptr[r + 1] - cptr[r]);
        else if (r >= gel_rows && r < gel_rows + 4 * nb) slots = std::max(slots, 4);
      }
      L.chunk_slots[ch] = slots;
      L.chunk_ptr[ch] = nblk;
      nblk += 32LL * slots;
    }
    L.n_blocks = nblk;
    L.sell_col.assign(nblk, 0);
    std::vector<int> cnt(nblk, 0);
    auto block_of = [&](int r, int sl) { return L.chunk_ptr[r / 32] + (long long)sl * 32 + (r % 32); };
    for (int ch = 0; ch < n_chunks; ++ch)
      for (int sl = 0; sl < L.chunk_slots[ch]; ++sl)
        for (int l = 0; l < 32; ++l) {
          int r = ch * 32 + l;
          int col = r;
          if (r < N) {
            if (sl < cptr[r + 1] - cptr[r]) col = cidx[cptr[r] + sl];
          } else if (r >= gel_rows && r < gel_rows + 4 * nb) {
            int b = (r - gel_rows) / 4;
            if (sl < 4) col = gel_rows + 4 * b + sl;
          }
          L.sell_col[L.chunk_ptr[ch] + (long long)sl * 32 + l] = col;
        }
    // contributions: tet block (a, b) -> SELL block of (row_a, row_b)
    std::vector<long long> dst(16 * (size_t)T);
    for (int t = 0; t < T; ++t)
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          int ra = L.tets[4 * t + a], rb = L.tets[4 * t + b];
          int sl;
          if (ra == rb) sl = 0;
          else sl = 1 + (int)(std::lower_bound(cidx.begin() + cptr[ra] + 1, cidx.begin() + cptr[ra + 1], rb) -
                              (cidx.begin() + cptr[ra] + 1));
          long long blk = block_of(ra, sl);
          dst[16 * (size_t)t + 4 * a + b] = blk;
          cnt[blk]++;
        }
    L.asm_ptr.assign(nblk + 1, 0);
    for (long long k = 0; k < nblk; ++k) L.asm_ptr[k + 1] = L.asm_ptr[k] + cnt[k];
    L.asm_src.resize(16 * (size_t)T);
    std::vector<int> fill(L.asm_ptr.begin(), L.asm_ptr.end() - 1);
    for (long long k = 0; k < 16LL * T; ++k) L.asm_src[fill[dst[k]]++] = (int)k;
    ev.n_chunks = n_chunks;
  }
  // ---------------- surface: boundary faces of the tet mesh (user ids, outward)
  std::vector<std::array<int, 3>> faces;
  {
    const int loc[4][3] = {{0, 2, 1}, {0, 1, 3}, {0, 3, 2}, {1, 2, 3}};
    std::vector<std::pair<std::array<int, 3>, std::array<int, 3>>> all;
    all.reserve(4 * (size_t)T);
    for (int t = 0; t < T; ++t)
      for (int f = 0; f < 4; ++f) {
        std::array<int, 3> tri = {s.tets[4 * t + loc[f][0]], s.tets[4 * t + loc[f][1]], s.tets[4 * t + loc[f][2]]};
        std::array<int, 3> key = tri;
        std::sort(key.begin(), key.end());
        all.push_back({key, tri});
      }
    std::sort(all.begin(), all.end());
    for (size_t i = 0; i < all.size();) {
      size_t j = i;
      while (j < all.size() && all[j].first == all[i].first) ++j;
      if (j - i == 1) faces.push_back(all[i].second);
      i = j;
    }
  }
  // ---------------- contact vertices: gel surface by pad, then body vertices
  std::vector<int> on_surf(N, 0);
  for (auto& f : faces) for (int v : f) on_surf[v] = 1;
  std::vector<int> gel_cv(N, -1);
  int ncv = 0;
  for (int p = 0; p < n_pads; ++p) {
    L.obj_cvb.push_back(ncv);
    for (int u = 0; u < N; ++u)
      if (on_surf[u] && pad[u] == p) {
        gel_cv[u] = ncv++;
        L.cv_row.push_back(ev.inv_perm[u]);
        L.cv_body.push_back(-1);
        L.cv_obj.push_back(p);
        L.cv_uid.push_back(u);
        L.cv_xbar.insert(L.cv_xbar.end(), {0.0, 0.0, 0.0});
        L.cv_fixed.push_back(pinned(u) ? 1 : 0);
      }
    L.obj_cve.push_back(ncv);
  }
  L.body_cv0.resize(nb);
  for (int b = 0; b < nb; ++b) {
    L.obj_cvb.push_back(ncv);
    L.body_cv0[b] = ncv;
    for (int j = 0; j < s.body_nv[b]; ++j) {
      ncv++;
      L.cv_row.push_back(gel_rows + 4 * b);
      L.cv_body.push_back(b);
      L.cv_obj.push_back(n_pads + b);
      L.cv_uid.push_back(N + bvoff[b] + j);
      for (int c = 0; c < 3; ++c) L.cv_xbar.push_back(s.body_rest_x[3 * (bvoff[b] + j) + c] - L.bp[b].com[c]);
      L.cv_fixed.push_back(0);
    }
    L.obj_cve.push_back(ncv);
  }
  ev.n_cv = ncv;
  std::vector<double> Xc(3 * (size_t)ncv);
  for (int i = 0; i < ncv; ++i) {
    int u = L.cv_uid[i];
    for (int c = 0; c < 3; ++c) Xc[3 * i + c] = (u < N) ? s.rest_x[3 * u + c] : s.body_rest_x[3 * (u - N) + c];
  }
  std::vector<std::vector<std::array<int, 3>>> otris(n_pads + nb);
  for (auto& f : faces) otris[pad[f[0]]].push_back({gel_cv[f[0]], gel_cv[f[1]], gel_cv[f[2]]});
  for (int b = 0; b < nb; ++b)
    for (int t = 0; t < s.body_nt[b]; ++t) {
      const int* q = s.body_tris + 3 * (btoff[b] + t);
      otris[n_pads + b].push_back({L.body_cv0[b] + q[0], L.body_cv0[b] + q[1], L.body_cv0[b] + q[2]});
    }
  L.cv_area.assign(ncv, 0.0);
  int ntri = 0, nedge = 0;
  for (int o = 0; o < n_pads + nb; ++o) {
    int tb = ntri;
    std::vector<std::pair<long long, double>> eareas;
    for (auto& t : otris[o]) {
      double a[3], b[3];
      for (int c = 0; c < 3; ++c) {
        a[c] = Xc[3 * t[1] + c] - Xc[3 * t[0] + c];
        b[c] = Xc[3 * t[2] + c] - Xc[3 * t[0] + c];
      }
      double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
      double ar = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
      for (int k = 0; k < 3; ++k) L.cv_area[t[k]] += ar / 3.0;
      for (int k = 0; k < 3; ++k) {
        int u = t[k], v = t[(k + 1) % 3];
        eareas.push_back({(long long)std::min(u, v) * ncv + std::max(u, v), ar / 3.0});
      }
      for (int k = 0; k < 3; ++k) L.tri.push_back(t[k]);
      L.tri_obj.push_back(o);
      ++ntri;
    }
    std::sort(eareas.begin(), eareas.end(),
              [](const std::pair<long long, double>& x, const std::pair<long long, double>& y) { return x.first < y.first; });
    int eb = nedge;
    for (size_t i = 0; i < eareas.size();) {
      size_t j = i;
      double ar = 0;
      while (j < eareas.size() && eareas[j].first == eareas[i].first) ar += eareas[j++].second;
      int u = (int)(eareas[i].first / ncv), v = (int)(eareas[i].first % ncv);
      L.edge.push_back(u);
      L.edge.push_back(v);
      L.edge_obj.push_back(o);
      L.edge_area.push_back(ar);
      double l2 = 0;
      for (int c = 0; c < 3; ++c) { double d = Xc[3 * u + c] - Xc[3 * v + c]; l2 += d * d; }
      L.edge_len2.push_back(l2);
      ++nedge;
      i = j;
    }
    L.obj_tb.push_back(tb);
    L.obj_te.push_back(ntri);
    L.obj_eb.push_back(eb);
    L.obj_ee.push_back(nedge);
    // an object never pairs with itself, except a pad flagged for
    // self-contact (its own primitives that share no vertex pair up)
    const bool self = o < n_pads && s.pad_self_contact && s.pad_self_contact[o];
    L.obj_ex.push_back(self ? 0ull : 1ull << o);
  }
  for (int u = 0; u < N; ++u)
    if (attach[u] >= 0) {
      int po = pad[u], bo = n_pads + attach[u];
      L.obj_ex[po] |= 1ull << bo;
      L.obj_ex[bo] |= 1ull << po;
    }
  ev.n_tri = ntri;
  ev.n_edge = nedge;
  ev.n_obj = n_pads + nb;
  // Morton orders of each object's points, triangles and edges at rest
  for (int o = 0; o < n_pads + nb; ++o) {
    std::vector<double> cen;
    for (int i = L.obj_cvb[o]; i < L.obj_cve[o]; ++i)
      for (int c = 0; c < 3; ++c) cen.push_back(Xc[3 * i + c]);
    morton_order(L.obj_cvb[o], L.obj_cve[o], cen, L.bv_ord[0]);
    cen.clear();
    for (int t = L.obj_tb[o]; t < L.obj_te[o]; ++t)
      for (int c = 0; c < 3; ++c)
        cen.push_back((Xc[3 * L.tri[3 * t] + c] + Xc[3 * L.tri[3 * t + 1] + c] + Xc[3 * L.tri[3 * t + 2] + c]) / 3.0);
    morton_order(L.obj_tb[o], L.obj_te[o], cen, L.bv_ord[1]);
    cen.clear();
    for (int q = L.obj_eb[o]; q < L.obj_ee[o]; ++q)
      for (int c = 0; c < 3; ++c) cen.push_back(0.5 * (Xc[3 * L.edge[2 * q] + c] + Xc[3 * L.edge[2 * q + 1] + c]));
    morton_order(L.obj_eb[o], L.obj_ee[o], cen, L.bv_ord[2]);
  }
  int nco = 0;
  for (int u = 0; u < N; ++u)
    if (on_surf[u] && !pinned(u) && attach[u] < 0) {
      L.coated_row.push_back(ev.inv_perm[u]);
      ++nco;
    }
  ev.n_coated = nco;
  ev.pair_cap = prm.max_pairs_per_env > 0 ? prm.max_pairs_per_env : 4 * ncv + 4096;
  return true;
}

template <class V>
void append_off(std::vector<V>& dst, const std::vector<V>& src, V off) {
  dst.reserve(dst.size() + src.size());
  for (const V& v : src) dst.push_back(v + off);
}
template <class V>
void append(std::vector<V>& dst, const std::vector<V>& src) {
  dst.insert(dst.end(), src.begin(), src.end());
}

}  // namespace

bool build_pack(const ipc_scene_desc* scenes, int n_envs, const ipc_params& prm, Pack& pk,
                std::string& err) {
  if (n_envs <= 0 || !scenes) { err = "n_envs must be positive"; return false; }
  pk = Pack();
  pk.n_envs = n_envs;
  pk.env.resize(n_envs);
  // pass 1: env-local builds (consecutive identical descriptors share one)
  std::vector<std::shared_ptr<EnvLocal>>& locals = pk.locals;
  locals.assign(n_envs, nullptr);
  for (int e = 0; e < n_envs; ++e) {
    if (e > 0 && std::memcmp(&scenes[e], &scenes[e - 1], sizeof(ipc_scene_desc)) == 0) {
      locals[e] = locals[e - 1];
      continue;
    }
    locals[e] = std::make_shared<EnvLocal>();
    if (!build_local(scenes[e], e, prm, *locals[e], err)) return false;
  }
  // reserve the flat tables
  {
    size_t R = 0, T = 0, CV = 0, TR = 0, ED = 0, OB = 0, BL = 0, CO = 0, CH = 0, AS = 0, NB = 0;
    for (auto& l : locals) {
      R += l->info.n_rows; T += l->info.n_tets; CV += l->info.n_cv; TR += l->info.n_tri; ED += l->info.n_edge;
      OB += l->info.n_obj; BL += l->n_blocks; CO += l->info.n_coated; CH += l->info.n_chunks;
      AS += l->asm_src.size(); NB += l->info.n_bodies;
    }
    pk.row_mass.reserve(R); pk.row_kind.reserve(R); pk.row_body.reserve(R); pk.row_xbar.reserve(3 * R);
    pk.rest_x.reserve(3 * R); pk.vt_ptr.reserve(R + 1); pk.vt_src.reserve(4 * T); pk.cta_env.reserve(R / 128);
    pk.tets.reserve(4 * T); pk.Dm_inv.reserve(9 * T); pk.tet_vol.reserve(T);
    pk.chunk_slots.reserve(CH); pk.chunk_ptr.reserve(CH); pk.sell_col.reserve(BL); pk.asm_ptr.reserve(BL + 1);
    pk.asm_src.reserve(AS);
    pk.cv_row.reserve(CV); pk.cv_body.reserve(CV); pk.cv_obj.reserve(CV); pk.cv_uid.reserve(CV);
    pk.cv_xbar.reserve(3 * CV); pk.cv_area.reserve(CV); pk.cv_fixed.reserve(CV);
    pk.tri.reserve(3 * TR); pk.tri_obj.reserve(TR); pk.edge.reserve(2 * ED); pk.edge_obj.reserve(ED);
    pk.edge_area.reserve(ED); pk.edge_len2.reserve(ED); pk.coated_row.reserve(CO);
    pk.body_S.reserve(9 * NB);
    (void)OB;
  }
  pk.asm_ptr.push_back(0);
  pk.vt_ptr.push_back(0);
  pk.env_row_off.push_back(0); pk.env_tet_off.push_back(0); pk.env_cv_off.push_back(0);
  pk.env_tri_off.push_back(0); pk.env_edge_off.push_back(0); pk.env_obj_off.push_back(0);
  pk.env_body_off.push_back(0); pk.env_chunk_off.push_back(0); pk.env_coated_off.push_back(0);
  pk.env_pair_off.push_back(0);
  for (int e = 0; e < n_envs; ++e) {
    const EnvLocal& L = *locals[e];
    EnvInfo ev = L.info;
    const int r0 = pk.env_row_off.back(), t0 = pk.env_tet_off.back(), c0 = pk.env_cv_off.back();
    const int tr0 = pk.env_tri_off.back(), e0 = pk.env_edge_off.back(), o0 = pk.env_obj_off.back();
    const int b0 = pk.env_body_off.back(), ch0 = pk.env_chunk_off.back(), co0 = pk.env_coated_off.back();
    const long long blk0 = pk.n_sell_blocks;
    ev.row_begin = r0; ev.tet_begin = t0; ev.cv_begin = c0; ev.tri_begin = tr0; ev.edge_begin = e0;
    ev.obj_begin = o0; ev.body_begin = b0; ev.chunk_begin = ch0; ev.coated_begin = co0;
    ev.pair_begin = pk.env_pair_off.back();
    const int R = ev.n_rows, T = ev.n_tets, nb = ev.n_bodies;
    for (int c = 0; c < R / 128; ++c) pk.cta_env.push_back(e);
    pk.env_mu.push_back(L.mu);
    pk.env_lam.push_back(L.lam);
    // rows
    append(pk.row_mass, L.row_mass);
    append(pk.row_kind, L.row_kind);
    for (int b : L.row_body) pk.row_body.push_back(b >= 0 ? b + b0 : -1);
    append(pk.row_xbar, L.row_xbar);
    append(pk.rest_x, L.rest_x);
    {
      int base = pk.vt_ptr.back();
      for (int r = 0; r < R; ++r) pk.vt_ptr.push_back(base + L.vt_ptr[r + 1]);
      append_off(pk.vt_src, L.vt_src, 4 * t0);
    }
    // tets
    append_off(pk.tets, L.tets, r0);
    append(pk.Dm_inv, L.Dm_inv);
    append(pk.tet_vol, L.vol);
    // SELL
    append(pk.chunk_slots, L.chunk_slots);
    append_off(pk.chunk_ptr, L.chunk_ptr, blk0);
    append_off(pk.sell_col, L.sell_col, r0);
    {
      int base = pk.asm_ptr.back();
      for (long long k = 0; k < L.n_blocks; ++k) pk.asm_ptr.push_back(base + L.asm_ptr[k + 1]);
      append_off(pk.asm_src, L.asm_src, 16 * t0);
    }
    pk.n_sell_blocks += L.n_blocks;
    // bodies
    for (int b = 0; b < nb; ++b) {
      pk.body_row.push_back(r0 + ev.gel_rows + 4 * b);
      pk.body_env.push_back(e);
      pk.body_cv_begin.push_back(c0 + L.body_cv0[b]);
      pk.body_nv.push_back(ev.body_nv[b]);
      pk.body_mass.push_back(L.bp[b].mass);
      pk.body_vol.push_back(L.bp[b].vol);
      pk.body_kappa.push_back(L.body_kappa[b]);
      pk.body_driven.push_back((uint8_t)L.body_driven[b]);
      for (int k = 0; k < 9; ++k) pk.body_S.push_back(L.bp[b].S[k]);
    }
    // contact
    append_off(pk.cv_row, L.cv_row, r0);
    for (int b : L.cv_body) pk.cv_body.push_back(b >= 0 ? b + b0 : -1);
    append_off(pk.cv_obj, L.cv_obj, o0);
    append(pk.cv_uid, L.cv_uid);
    append(pk.cv_xbar, L.cv_xbar);
    append(pk.cv_area, L.cv_area);
    append(pk.cv_fixed, L.cv_fixed);
    append_off(pk.tri, L.tri, c0);
    append_off(pk.tri_obj, L.tri_obj, o0);
    append_off(pk.edge, L.edge, c0);
    append_off(pk.edge_obj, L.edge_obj, o0);
    append(pk.edge_area, L.edge_area);
    append(pk.edge_len2, L.edge_len2);
    for (int o = 0; o < ev.n_obj; ++o) {
      pk.obj_env.push_back(e);
      pk.obj_local.push_back(o);
      pk.obj_cv_begin.push_back(c0 + L.obj_cvb[o]);
      pk.obj_cv_end.push_back(c0 + L.obj_cve[o]);
      pk.obj_tri_begin.push_back(tr0 + L.obj_tb[o]);
      pk.obj_tri_end.push_back(tr0 + L.obj_te[o]);
      pk.obj_edge_begin.push_back(e0 + L.obj_eb[o]);
      pk.obj_edge_end.push_back(e0 + L.obj_ee[o]);
      pk.obj_size.push_back((L.obj_cve[o] - L.obj_cvb[o]) + (L.obj_te[o] - L.obj_tb[o]) + (L.obj_ee[o] - L.obj_eb[o]));
      pk.obj_exclude.push_back(L.obj_ex[o]);
    }
    append_off(pk.coated_row, L.coated_row, r0);
    // broad-phase hierarchy: Morton-ordered primitives, clusters of 32 and
    // superclusters of 32 clusters per object and kind
    {
      const int pofs[3] = {c0, tr0, e0};
      append_off(pk.bv_perm[0], L.bv_ord[0], c0);
      append_off(pk.bv_perm[1], L.bv_ord[1], tr0);
      append_off(pk.bv_perm[2], L.bv_ord[2], e0);
      for (int o = 0; o < ev.n_obj; ++o) {
        const int np[3] = {L.obj_cve[o] - L.obj_cvb[o], L.obj_te[o] - L.obj_tb[o], L.obj_ee[o] - L.obj_eb[o]};
        for (int k = 0; k < 3; ++k) {
          const int ncl = (np[k] + 31) / 32, nsc = (ncl + 31) / 32;
          pk.obj_cl_begin[k].push_back((int)pk.bv_cl_obj[k].size());
          pk.obj_sc_begin[k].push_back((int)pk.bv_sc_obj[k].size());
          for (int j = 0; j < ncl; ++j) pk.bv_cl_obj[k].push_back(o0 + o);
          for (int j = 0; j < nsc; ++j) pk.bv_sc_obj[k].push_back(o0 + o);
        }
      }
      (void)pofs;
    }

    pk.env[e] = ev;
    pk.env_row_off.push_back(r0 + R);
    pk.env_tet_off.push_back(t0 + T);
    pk.env_cv_off.push_back(c0 + ev.n_cv);
    pk.env_tri_off.push_back(tr0 + ev.n_tri);
    pk.env_edge_off.push_back(e0 + ev.n_edge);
    pk.env_obj_off.push_back(o0 + ev.n_obj);
    pk.env_body_off.push_back(b0 + nb);
    pk.env_chunk_off.push_back(ch0 + ev.n_chunks);
    pk.env_coated_off.push_back(co0 + ev.n_coated);
    pk.env_pair_off.push_back(ev.pair_begin + ev.pair_cap);
    pk.env_pair_cap.push_back(ev.pair_cap);
  }
  pk.n_rows = pk.env_row_off.back();
  pk.n_tets = pk.env_tet_off.back();
  pk.n_cv = pk.env_cv_off.back();
  pk.n_tri = pk.env_tri_off.back();
  pk.n_edge = pk.env_edge_off.back();
  pk.n_obj = pk.env_obj_off.back();
  pk.n_bodies = pk.env_body_off.back();
  pk.n_chunks = pk.env_chunk_off.back();
  pk.n_coated = pk.env_coated_off.back();
  pk.n_pairs_cap = pk.env_pair_off.back();
  return true;
}

bool build_env_local(const ipc_scene_desc& s, int e, const ipc_params& prm, std::shared_ptr<EnvLocal>& out,
                     std::string& err) {
  out = std::make_shared<EnvLocal>();
  return build_local(s, e, prm, *out, err);
}

// Equal topology: every index table and count that fixes the layout of the
// env's segments in the flat tables (rows, SELL pattern, contact primitives,
// objects, coated rows).  Values that may differ: material, masses, rest
// geometry, body mass properties, contact areas and rest edge lengths.
bool same_topology(const EnvLocal& a, const EnvLocal& b) {
  const EnvInfo &x = a.info, &y = b.info;
  if (x.n_verts != y.n_verts || x.n_tets != y.n_tets || x.n_bodies != y.n_bodies || x.n_pads != y.n_pads ||
      x.n_rows != y.n_rows || x.gel_rows != y.gel_rows || x.n_cv != y.n_cv || x.n_tri != y.n_tri ||
      x.n_edge != y.n_edge || x.n_obj != y.n_obj || x.n_chunks != y.n_chunks || x.n_coated != y.n_coated ||
      x.pair_cap != y.pair_cap || x.perm != y.perm || x.body_nv != y.body_nv)
    return false;
  return a.row_kind == b.row_kind && a.row_body == b.row_body && a.vt_ptr == b.vt_ptr && a.vt_src == b.vt_src &&
         a.tets == b.tets && a.chunk_slots == b.chunk_slots && a.chunk_ptr == b.chunk_ptr &&
         a.sell_col == b.sell_col && a.asm_ptr == b.asm_ptr && a.asm_src == b.asm_src && a.n_blocks == b.n_blocks &&
         a.body_cv0 == b.body_cv0 && a.cv_row == b.cv_row && a.cv_body == b.cv_body && a.cv_obj == b.cv_obj &&
         a.cv_uid == b.cv_uid && a.tri == b.tri && a.tri_obj == b.tri_obj && a.edge == b.edge &&
         a.edge_obj == b.edge_obj && a.obj_cvb == b.obj_cvb && a.obj_cve == b.obj_cve && a.obj_tb == b.obj_tb &&
         a.obj_te == b.obj_te && a.obj_eb == b.obj_eb && a.obj_ee == b.obj_ee && a.obj_ex == b.obj_ex &&
         a.coated_row == b.coated_row;
}

// Writes env e's value tables of L into the flat host tables (same
// topology as the env's current local build).
void patch_env_values(Pack& pk, int e, const EnvLocal& L) {
  EnvInfo& ev = pk.env[e];
  const int r0 = ev.row_begin, t0 = ev.tet_begin, c0 = ev.cv_begin, b0 = ev.body_begin;
  const int tr0 = ev.tri_begin, e0 = ev.edge_begin;
  pk.env_mu[e] = L.mu;
  pk.env_lam[e] = L.lam;
  std::copy(L.row_mass.begin(), L.row_mass.end(), pk.row_mass.begin() + r0);
  std::copy(L.row_xbar.begin(), L.row_xbar.end(), pk.row_xbar.begin() + 3 * (size_t)r0);
  std::copy(L.rest_x.begin(), L.rest_x.end(), pk.rest_x.begin() + 3 * (size_t)r0);
  std::copy(L.Dm_inv.begin(), L.Dm_inv.end(), pk.Dm_inv.begin() + 9 * (size_t)t0);
  std::copy(L.vol.begin(), L.vol.end(), pk.tet_vol.begin() + t0);
  for (int b = 0; b < ev.n_bodies; ++b) {
    pk.body_mass[b0 + b] = L.bp[b].mass;
    pk.body_vol[b0 + b] = L.bp[b].vol;
    pk.body_kappa[b0 + b] = L.body_kappa[b];
    pk.body_driven[b0 + b] = (uint8_t)L.body_driven[b];
    for (int k = 0; k < 9; ++k) pk.body_S[9 * (size_t)(b0 + b) + k] = L.bp[b].S[k];
  }
  std::copy(L.cv_xbar.begin(), L.cv_xbar.end(), pk.cv_xbar.begin() + 3 * (size_t)c0);
  std::copy(L.cv_area.begin(), L.cv_area.end(), pk.cv_area.begin() + c0);
  std::copy(L.cv_fixed.begin(), L.cv_fixed.end(), pk.cv_fixed.begin() + c0);
  std::copy(L.edge_area.begin(), L.edge_area.end(), pk.edge_area.begin() + e0);
  std::copy(L.edge_len2.begin(), L.edge_len2.end(), pk.edge_len2.begin() + e0);
  const int off[3] = {c0, tr0, e0};
  for (int k = 0; k < 3; ++k)
    for (size_t i = 0; i < L.bv_ord[k].size(); ++i) pk.bv_perm[k][off[k] + i] = L.bv_ord[k][i] + off[k];
  ev.body_com = L.info.body_com;
  pk.locals[e] = std::make_shared<EnvLocal>(L);
}

}  // namespace ipc
