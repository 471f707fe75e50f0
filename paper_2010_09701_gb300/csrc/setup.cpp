// Host-side geometry: 1D rules, periodic spectral-element mesh, enrichment
// supports and the per-cell quadrature point sets (Sec. III A and III B).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <set>

#include "oefe_internal.h"

// ------------------------------------------------------------------ 1D rules
static void legendre(int n, double x, double* P, double* dP) {
  // P_n(x) and P_n'(x) by the three-term recurrence
  double p0 = 1.0, p1 = x;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  // derivative from n (x P_n - P_{n-1}) / (x^2 - 1), valid away from +-1
  *dP = n * (x * p1 - p0) / (x * x - 1.0);
}

void gll_rule(int p, std::vector<double>& x, std::vector<double>& w) {
  // nodes: -1, 1 and the roots of P_p'; weights 2 / (p (p+1) P_p(x)^2)
  x.assign(p + 1, 0.0);
  w.assign(p + 1, 0.0);
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double t = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, t, &P, &dP);
      // Legendre ODE: (1 - t^2) P'' = 2 t P' - p (p+1) P
      double d2P = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
      double dt = dP / d2P;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
  std::sort(x.begin(), x.end());
  for (int i = 0; i <= p; ++i) {
    double P, dP;
    legendre(p, x[i], &P, &dP);
    if (i == 0 || i == p) P = (i == 0 && (p % 2)) ? -1.0 : 1.0;
    w[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
}

void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double P = 0, dP = 1;
    for (int it = 0; it < 100; ++it) {
      legendre(n, t, &P, &dP);
      double dt = P / dP;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    legendre(n, t, &P, &dP);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
  // ascending order
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return x[a] < x[b]; });
  std::vector<double> xs(n), ws(n);
  for (int i = 0; i < n; ++i) { xs[i] = x[idx[i]]; ws[i] = w[idx[i]]; }
  x = xs;
  w = ws;
}

// ------------------------------------------------------------------ helpers
int dev_alloc(oefe_ctx* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    c->err = std::string("device allocation of ") + std::to_string(bytes) + " bytes failed: " +
             cudaGetErrorString(e);
    cudaGetLastError();
    return OEFE_ERR_OOM;
  }
  return OEFE_OK;
}

void dev_free(void* p) {
  if (p) cudaFree(p);
}

int ensure_ws(oefe_ctx* c, size_t bytes) {
  if (bytes <= c->ws_bytes) return OEFE_OK;
  cudaStreamSynchronize(c->stream);
  dev_free(c->ws);
  c->ws = nullptr;
  c->ws_bytes = 0;
  OEFE_TRY(dev_alloc(c, &c->ws, bytes));
  c->ws_bytes = bytes;
  return OEFE_OK;
}

int ensure_ws2(oefe_ctx* c, size_t bytes) {
  if (bytes <= c->ws2_bytes) return OEFE_OK;
  cudaStreamSynchronize(c->stream);
  dev_free(c->ws2);
  c->ws2 = nullptr;
  c->ws2_bytes = 0;
  OEFE_TRY(dev_alloc(c, &c->ws2, bytes));
  c->ws2_bytes = bytes;
  return OEFE_OK;
}

template <typename T>
static int upload(oefe_ctx* c, T** d, const std::vector<T>& h) {
  dev_free(*d);
  *d = nullptr;
  OEFE_TRY(dev_alloc(c, (void**)d, h.size() * sizeof(T)));
  if (!h.empty())
    OEFE_CUDA_TRY(c, cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice,
                                     c->stream));
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return OEFE_OK;
}

// ------------------------------------------------------------------ mesh
int setup_mesh(oefe_ctx* c, double a, const int ncell[3], const double* xb, int p) {
  if (!(a > 0) || p < 1 || p > 7 || !xb) { c->err = "mesh: need a > 0, 1 <= p <= 7, xb"; return OEFE_ERR_ARG; }
  int off = 0;
  for (int d = 0; d < 3; ++d) {
    if (ncell[d] < 1 || ncell[d] > 4096) { c->err = "mesh: ncell out of range"; return OEFE_ERR_ARG; }
    c->xb[d].assign(xb + off, xb + off + ncell[d] + 1);
    off += ncell[d] + 1;
    if (c->xb[d][0] != 0.0 || std::fabs(c->xb[d].back() - a) > 1e-12 * a) {
      c->err = "mesh: breakpoints must run from 0 to a";
      return OEFE_ERR_ARG;
    }
    for (int i = 0; i < ncell[d]; ++i)
      if (!(c->xb[d][i + 1] > c->xb[d][i])) { c->err = "mesh: breakpoints must increase"; return OEFE_ERR_ARG; }
    c->nc[d] = ncell[d];
  }
  c->a = a;
  c->p = p;
  c->P = p + 1;
  c->nloc = c->P * c->P * c->P;
  for (int d = 0; d < 3; ++d) c->N[d] = c->nc[d] * p;
  c->nh = (int64_t)c->N[0] * c->N[1] * c->N[2];
  c->ncells = c->nc[0] * c->nc[1] * c->nc[2];
  if (c->nh > (int64_t)1 << 31) { c->err = "mesh: more than 2^31 nodes"; return OEFE_ERR_ARG; }
  gll_rule(p, c->gll_x, c->gll_w);

  const int P = c->P;
  c->cell_nodes.assign((size_t)c->ncells * c->nloc, 0);
  std::vector<double> m(c->nh, 0.0), box((size_t)c->ncells * 6);
  for (int e = 0; e < c->ncells; ++e) {
    int ix = e % c->nc[0], iy = (e / c->nc[0]) % c->nc[1], iz = e / (c->nc[0] * c->nc[1]);
    double lo[3] = {c->xb[0][ix], c->xb[1][iy], c->xb[2][iz]};
    double h[3] = {c->xb[0][ix + 1] - lo[0], c->xb[1][iy + 1] - lo[1], c->xb[2][iz + 1] - lo[2]};
    for (int d = 0; d < 3; ++d) { box[6 * e + d] = lo[d]; box[6 * e + 3 + d] = h[d]; }
    double vol8 = h[0] * h[1] * h[2] / 8.0;
    for (int k = 0; k < P; ++k)
      for (int j = 0; j < P; ++j)
        for (int i = 0; i < P; ++i) {
          int gx = (ix * p + i) % c->N[0], gy = (iy * p + j) % c->N[1], gz = (iz * p + k) % c->N[2];
          int g = gx + c->N[0] * (gy + c->N[1] * gz);
          c->cell_nodes[(size_t)e * c->nloc + i + P * (j + P * k)] = g;
          m[g] += c->gll_w[i] * c->gll_w[j] * c->gll_w[k] * vol8;
        }
  }
  OEFE_TRY(upload(c, &c->d_m, m));
  OEFE_TRY(upload(c, &c->d_cell_nodes, c->cell_nodes));
  OEFE_TRY(upload(c, &c->d_cellbox, box));
  OEFE_TRY(upload(c, &c->d_gll, c->gll_x));
  c->has_mesh = true;
  c->has_enr = c->has_quad = c->has_k = c->built = false;
  return OEFE_OK;
}

void graded_breakpoints(double a, int ncell, const std::vector<double>& coords, double ratio,
                        std::vector<double>& out) {
  const double tol = 1e-3;
  std::vector<double> cs;
  for (double x : coords) cs.push_back(x - a * std::floor(x / a));
  std::sort(cs.begin(), cs.end());
  std::vector<double> uq;
  for (double x : cs)
    if (uq.empty() || x - uq.back() > tol) uq.push_back(x);
  if (uq.size() > 1 && (uq[0] + a) - uq.back() <= tol) uq.pop_back();
  out.clear();
  if (uq.empty() || (int)uq.size() > ncell / 2) {
    for (int i = 0; i <= ncell; ++i) out.push_back(a * i / ncell);
    return;
  }
  if (uq[0] > tol) uq.insert(uq.begin(), 0.0);
  std::vector<double> ends = uq;
  ends.push_back(a);
  int nint = (int)uq.size();
  std::vector<double> len(nint), share(nint), rem(nint);
  std::vector<int> cnt(nint);
  for (int i = 0; i < nint; ++i) {
    len[i] = ends[i + 1] - ends[i];
    share[i] = len[i] / a * ncell;
    cnt[i] = std::max((int)std::floor(share[i]), 2);
    rem[i] = share[i] - std::floor(share[i]);
  }
  auto total = [&]() { int s = 0; for (int v : cnt) s += v; return s; };
  while (total() > ncell) {
    int j = 0;
    for (int i = 1; i < nint; ++i)
      if (cnt[i] - share[i] > cnt[j] - share[j]) j = i;
    cnt[j] -= 1;
  }
  while (total() < ncell) {
    int j = 0;
    for (int i = 1; i < nint; ++i)
      if (rem[i] > rem[j]) j = i;
    cnt[j] += 1;
    rem[j] = -1;
  }
  out.push_back(0.0);
  for (int i = 0; i < nint; ++i) {
    int n = cnt[i];
    std::vector<double> half, wv;
    for (int j = 0; j < (n + 1) / 2; ++j) half.push_back(std::pow(ratio, j));
    wv = half;
    for (int j = (int)half.size() - 1 - (n % 2); j >= 0; --j) wv.push_back(half[j]);
    double s = 0;
    for (double v : wv) s += v;
    double acc = ends[i];
    for (size_t j = 0; j + 1 < wv.size(); ++j) {
      acc += wv[j] / s * len[i];
      out.push_back(acc);
    }
    out.push_back(ends[i] + len[i]);
  }
  out.back() = a;
}

// ------------------------------------------------------------------ supports
static double box_point_dist2(const double lo[3], const double hi[3], const double R[3], double a) {
  double s = 0;
  for (int d = 0; d < 3; ++d) {
    double best = 1e300;
    for (int n = -1; n <= 1; ++n) {
      double y = R[d] + n * a;
      double t = std::max(std::max(lo[d] - y, 0.0), y - hi[d]);
      best = std::min(best, t);
    }
    s += best * best;
  }
  return s;
}

static bool box_holds_point(const double lo[3], const double hi[3], const double R[3], double a) {
  double tol = 1e-12 * a;
  for (int d = 0; d < 3; ++d) {
    bool any = false;
    for (int n = -1; n <= 1; ++n) {
      double y = R[d] + n * a;
      if (lo[d] - tol <= y && y <= hi[d] + tol) any = true;
    }
    if (!any) return false;
  }
  return true;
}

void cell_box(const oefe_ctx* c, int e, double lo[3], double hi[3]) {
  int ix = e % c->nc[0], iy = (e / c->nc[0]) % c->nc[1], iz = e / (c->nc[0] * c->nc[1]);
  lo[0] = c->xb[0][ix]; hi[0] = c->xb[0][ix + 1];
  lo[1] = c->xb[1][iy]; hi[1] = c->xb[1][iy + 1];
  lo[2] = c->xb[2][iz]; hi[2] = c->xb[2][iz + 1];
}

int setup_enrichment(oefe_ctx* c, int natoms, const double* pos, int nfun, const int* lm, int ngrid,
                     const double* R, const double* dR, double r0, double rc) {
  if (!c->has_mesh) { c->err = "enrichment: call oefe_mesh first"; return OEFE_ERR_STATE; }
  if (natoms < 0 || nfun < 0 || (natoms > 0 && nfun == 0) || (natoms > 0 && (!pos || !lm || !R || !dR)) ||
      !(r0 > 0) || !(rc > r0) || !(rc < 0.5 * c->a) || (natoms > 0 && ngrid < 4)) {
    c->err = "enrichment: need natoms >= 0, nfun >= 1, ngrid >= 4, 0 < r0 < rc < a/2";
    return OEFE_ERR_ARG;
  }
  for (int j = 0; j < nfun; ++j)
    if (lm[j] < 0 || lm[j] > 3) { c->err = "enrichment: lm codes must be 0..3"; return OEFE_ERR_ARG; }
  if (natoms * nfun > 4096) { c->err = "enrichment: at most 4096 functions"; return OEFE_ERR_ARG; }
  c->natoms = natoms;
  c->nfun = natoms > 0 ? nfun : 0;
  c->nO = natoms * c->nfun;
  c->ngrid = ngrid;
  c->r0 = r0;
  c->rc = rc;
  c->pos.assign(pos, pos + 3 * natoms);
  c->lm.assign(lm, lm + c->nfun);
  std::vector<double> Rv, dRv;
  if (natoms > 0) {
    Rv.assign(R, R + (size_t)natoms * nfun * ngrid);
    dRv.assign(dR, dR + (size_t)natoms * nfun * ngrid);
  }
  OEFE_TRY(upload(c, &c->d_R, Rv));
  OEFE_TRY(upload(c, &c->d_dR, dRv));
  OEFE_TRY(upload(c, &c->d_pos, c->pos));
  OEFE_TRY(upload(c, &c->d_lm, c->lm));

  // act_A(e): atoms whose ball meets the cell; act(e): union over the 27 neighbours
  const int nc = c->ncells;
  std::vector<std::vector<int>> actA(nc);
  for (int e = 0; e < nc; ++e) {
    double lo[3], hi[3];
    cell_box(c, e, lo, hi);
    for (int I = 0; I < natoms; ++I)
      if (box_point_dist2(lo, hi, &c->pos[3 * I], c->a) < rc * rc) actA[e].push_back(I);
  }
  c->act_off.assign(nc + 1, 0);
  c->act_idx.clear();
  c->ne_max = 0;
  for (int e = 0; e < nc; ++e) {
    int ix = e % c->nc[0], iy = (e / c->nc[0]) % c->nc[1], iz = e / (c->nc[0] * c->nc[1]);
    std::set<int> atoms;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int jx = (ix + dx + c->nc[0]) % c->nc[0], jy = (iy + dy + c->nc[1]) % c->nc[1],
              jz = (iz + dz + c->nc[2]) % c->nc[2];
          for (int I : actA[jx + c->nc[0] * (jy + c->nc[1] * jz)]) atoms.insert(I);
        }
    for (int I : atoms)
      for (int j = 0; j < c->nfun; ++j) c->act_idx.push_back(I * c->nfun + j);
    c->act_off[e + 1] = (int)c->act_idx.size();
    c->ne_max = std::max(c->ne_max, c->act_off[e + 1] - c->act_off[e]);
  }
  c->npad = ((c->nloc + c->ne_max + 127) / 128) * 128;
  OEFE_TRY(upload(c, &c->d_act_off, c->act_off));
  OEFE_TRY(upload(c, &c->d_act_idx, c->act_idx));

  // node -> slots
  std::vector<int64_t> noff(c->nh + 1, 0), nslot((size_t)nc * c->nloc);
  for (int e = 0; e < nc; ++e)
    for (int l = 0; l < c->nloc; ++l) noff[c->cell_nodes[(size_t)e * c->nloc + l] + 1]++;
  for (int64_t i = 0; i < c->nh; ++i) noff[i + 1] += noff[i];
  {
    std::vector<int64_t> fill(noff.begin(), noff.end() - 1);
    for (int e = 0; e < nc; ++e)
      for (int l = 0; l < c->nloc; ++l) {
        int g = c->cell_nodes[(size_t)e * c->nloc + l];
        nslot[fill[g]++] = (int64_t)e * c->npad + l;
      }
  }
  OEFE_TRY(upload(c, &c->d_node_off, noff));
  OEFE_TRY(upload(c, &c->d_node_slot, nslot));
  // enrichment function -> slots
  std::vector<int64_t> eoff(c->nO + 1, 0), eslot;
  for (int e = 0; e < nc; ++e)
    for (int j = c->act_off[e]; j < c->act_off[e + 1]; ++j) eoff[c->act_idx[j] + 1]++;
  for (int i = 0; i < c->nO; ++i) eoff[i + 1] += eoff[i];
  eslot.assign(eoff[c->nO], 0);
  {
    std::vector<int64_t> fill(eoff.begin(), eoff.end() - 1);
    for (int e = 0; e < nc; ++e)
      for (int j = c->act_off[e]; j < c->act_off[e + 1]; ++j)
        eslot[fill[c->act_idx[j]]++] = (int64_t)e * c->npad + c->nloc + (j - c->act_off[e]);
  }
  c->enr_off_h = eoff;
  OEFE_TRY(upload(c, &c->d_enr_off, eoff));
  OEFE_TRY(upload(c, &c->d_enr_slot, eslot));
  c->has_enr = true;
  c->has_quad = c->has_k = c->built = false;
  return OEFE_OK;
}

// ------------------------------------------------------------------ quadrature
static void make_leaves(const oefe_ctx* c, const double lo[3], const double hi[3], int level,
                        std::vector<std::pair<std::array<double, 3>, std::array<double, 3>>>& out) {
  bool holds = false;
  for (int I = 0; I < c->natoms && !holds; ++I) holds = box_holds_point(lo, hi, &c->pos[3 * I], c->a);
  if (level < c->depth && holds) {
    double mid[3];
    for (int d = 0; d < 3; ++d) mid[d] = 0.5 * (lo[d] + hi[d]);
    for (int cz = 0; cz < 2; ++cz)
      for (int cy = 0; cy < 2; ++cy)
        for (int cx = 0; cx < 2; ++cx) {
          int cc[3] = {cx, cy, cz};
          double clo[3], chi[3];
          for (int d = 0; d < 3; ++d) {
            clo[d] = cc[d] == 0 ? lo[d] : mid[d];
            chi[d] = cc[d] == 0 ? mid[d] : hi[d];
          }
          make_leaves(c, clo, chi, level + 1, out);
        }
    return;
  }
  out.push_back({{lo[0], lo[1], lo[2]}, {hi[0], hi[1], hi[2]}});
}

int setup_quadrature(oefe_ctx* c, int nq_cell, int nq_enr, int depth) {
  if (!c->has_enr) { c->err = "quadrature: call oefe_enrichment first"; return OEFE_ERR_STATE; }
  if (nq_cell < 1 || nq_cell > 12 || nq_enr < 1 || nq_enr > 12 || depth < 0 || depth > 12) {
    c->err = "quadrature: 1 <= nq <= 12, 0 <= depth <= 12";
    return OEFE_ERR_ARG;
  }
  c->nq_cell = nq_cell;
  c->nq_enr = nq_enr;
  dev_free(c->d_veff);   // sized by the point count
  c->d_veff = nullptr;
  c->depth = depth;
  c->leaves.clear();
  c->leaf_off.assign(c->ncells + 1, 0);
  c->q_off.assign(c->ncells + 1, 0);
  c->qxyz.clear();
  c->qw.clear();
  std::vector<double> gx[13], gw[13];
  for (int n : {nq_cell, nq_enr}) gauss_rule(n, gx[n], gw[n]);
  int64_t q = 0;
  for (int e = 0; e < c->ncells; ++e) {
    double lo[3], hi[3];
    cell_box(c, e, lo, hi);
    int cls = 0;
    for (int I = 0; I < c->natoms; ++I)
      if (box_holds_point(lo, hi, &c->pos[3 * I], c->a)) cls = 2;
    if (cls == 0)
      for (int I = 0; I < c->natoms; ++I)
        if (box_point_dist2(lo, hi, &c->pos[3 * I], c->a) < c->rc * c->rc) cls = 1;
    std::vector<std::pair<std::array<double, 3>, std::array<double, 3>>> lv;
    if (cls == 2) make_leaves(c, lo, hi, 0, lv);
    else lv.push_back({{lo[0], lo[1], lo[2]}, {hi[0], hi[1], hi[2]}});
    int n = cls == 0 ? nq_cell : nq_enr;
    const std::vector<double>& t = gx[n];
    const std::vector<double>& w = gw[n];
    double h[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    for (auto& b : lv) {
      Leaf L;
      L.cell = e;
      L.n1 = n;
      L.q0 = q;
      for (int d = 0; d < 3; ++d) {
        L.lo[d] = b.first[d];
        L.hi[d] = b.second[d];
      }
      c->leaves.push_back(L);
      double dx = b.second[0] - b.first[0], dy = b.second[1] - b.first[1], dz = b.second[2] - b.first[2];
      double vol8 = dx * dy * dz / 8.0;
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            c->qxyz.push_back(b.first[0] + (t[i] + 1) / 2 * dx);
            c->qxyz.push_back(b.first[1] + (t[j] + 1) / 2 * dy);
            c->qxyz.push_back(b.first[2] + (t[k] + 1) / 2 * dz);
            c->qw.push_back(w[i] * w[j] * w[k] * vol8);
            ++q;
          }
    }
    (void)h;
    c->leaf_off[e + 1] = (int)c->leaves.size();
    c->q_off[e + 1] = q;
  }
  c->nq = q;
  OEFE_TRY(upload(c, &c->d_qxyz, c->qxyz));
  OEFE_TRY(upload(c, &c->d_qw, c->qw));
  OEFE_TRY(upload(c, &c->d_leaves, c->leaves));
  OEFE_TRY(upload(c, &c->d_leaf_off, c->leaf_off));
  OEFE_TRY(upload(c, &c->d_q_off, c->q_off));
  OEFE_TRY(setup_sumfac(c));
  c->has_quad = true;
  c->has_k = c->built = false;
  return OEFE_OK;
}
