// Host side of the C ABI declared in include/gpeps.h: graph validation, edge
// colouring, per-colour bond work lists, caller-owned buffer layout, launches
// and the per-step CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "gpeps.h"
#include "gpeps_internal.cuh"

using namespace gpeps;

namespace {

thread_local std::string g_last_cuda;

int cuda_fail(cudaError_t e, const char* where) {
  g_last_cuda = std::string(where) + ": " + cudaGetErrorString(e);
  return GPEPS_ECUDA;
}

#define GP_CUDA(call)                                       \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct ColourPlan {
  std::vector<BondDesc> bonds;
  std::vector<TileDesc> tiles;
  size_t w_bonds = 0, w_tiles = 0;  // byte offsets in the work buffer
  int n_parts = 0;
};

struct InstGraph {
  int n = 0;
  std::vector<std::pair<int, int>> edges;  // as given
  std::vector<int> colour;
  std::vector<std::vector<int>> nb;        // sorted neighbours
  std::vector<std::vector<int>> nb_edge;   // edge index of each neighbour
};

int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

}  // namespace

struct gpeps_handle {
  int D = 0, dtype = 0, n_inst = 0;
  size_t elt = 0;  // bytes per complex element
  cudaStream_t stream = nullptr;
  std::vector<InstGraph> g;
  int64_t total_sites = 0, total_edges = 0;
  std::vector<int32_t> inst_site0, inst_edge0, site_inst;
  std::vector<int64_t> site_off;
  std::vector<SiteDesc> sites;
  int64_t n_gamma = 0;  // complex elements of all Gamma
  std::vector<ColourPlan> colours;
  int max_parts = 0, max_bonds = 0;
  JacobiParams jp{};
  // buffer layout (bytes)
  size_t state_bytes = 0, work_bytes = 0;
  size_t s_lam = 0, s_gamma = 0;
  size_t w_pending = 0, w_flags = 0, w_sweeps = 0, w_cycles = 0, w_queue = 0, w_z = 0, w_mean = 0, w_sites = 0, w_inst_site0 = 0,
         w_site_inst = 0, w_site_off = 0, w_partials = 0, w_Y = 0, w_theta_a = 0, w_bond_scratch = 0;
  size_t bond_slot = 0;  // bytes per bond-kernel CTA of global scratch for its n x n matrices
  int bond_slots = 0;    // slots in the work buffer
  char* d_state = nullptr;
  char* d_work = nullptr;
  bool bound = false;
  bool tensor = false;  // mixed path, D = 32 or 64: Gram and update passes of the larger ends on the tensor cores
  int schedule = 0;  // bond eigenproblems: 0 one CTA per bond; work queue with 1 (schedule 1), 2 (2) or 4 (3)
                     // CTAs per SM; 4 fused step (gpeps_step: one persistent launch over every colour class);
                     // 5 and 6 the fused step with three or four CTAs per SM
  std::vector<StepTask> tasks;  // fused step: every bond of a step, colour by colour, with its dependencies
  // BP regauging: half-edges (one per leg of every site), work lists built on first use
  int64_t n_half = 0;
  std::vector<int32_t> he0;  // half-edge index of leg 0 of every site
  std::vector<BpMsgTask> bp_msgs;
  std::vector<BpEdgeTask> bp_edges;
  std::vector<BpSiteTask> bp_sites;
  size_t w_tasks = 0, w_done = 0;
  int n_sms = 0;
  int64_t bonds_since_reset = 0;
  // captured step
  cudaGraphExec_t step_exec = nullptr;
  const double* step_theta = nullptr;
  int step_per_qubit = -1;

  double* lam() const { return reinterpret_cast<double*>(d_state + s_lam); }
  void* gamma() const { return d_state + s_gamma; }
  double* pending() const { return reinterpret_cast<double*>(d_work + w_pending); }
  int* flags() const { return reinterpret_cast<int*>(d_work + w_flags); }
  unsigned long long* sweeps() const { return reinterpret_cast<unsigned long long*>(d_work + w_sweeps); }
  unsigned long long* cycles() const { return reinterpret_cast<unsigned long long*>(d_work + w_cycles); }
  double* z() const { return reinterpret_cast<double*>(d_work + w_z); }
  double* mean() const { return reinterpret_cast<double*>(d_work + w_mean); }
  template <typename P>
  P* at(size_t off) const {
    return reinterpret_cast<P*>(d_work + off);
  }
};

namespace {

int validate_and_colour(const gpeps_graph& gr, InstGraph& ig) {
  if (gr.n_qubits < 1 || gr.n_edges < 0) return GPEPS_EINVAL;
  if (gr.n_edges > 0 && gr.edges == nullptr) return GPEPS_EINVAL;
  ig.n = gr.n_qubits;
  ig.nb.assign(ig.n, {});
  ig.edges.resize(gr.n_edges);
  std::vector<std::pair<int, int>> seen;
  seen.reserve(gr.n_edges);
  for (int e = 0; e < gr.n_edges; ++e) {
    const int a = gr.edges[2 * e], b = gr.edges[2 * e + 1];
    if (a < 0 || b < 0 || a >= ig.n || b >= ig.n || a == b) return GPEPS_EINVAL;
    ig.edges[e] = {a, b};
    seen.emplace_back(std::min(a, b), std::max(a, b));
    ig.nb[a].push_back(b);
    ig.nb[b].push_back(a);
  }
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return GPEPS_EINVAL;
  for (int v = 0; v < ig.n; ++v) {
    if (ig.nb[v].size() > 3) return GPEPS_EINVAL;
    std::sort(ig.nb[v].begin(), ig.nb[v].end());
  }
  for (auto& e : ig.edges)
    if (ig.nb[e.first].size() == 3 && ig.nb[e.second].size() == 3) return GPEPS_EINVAL;
  // edge index of each leg
  ig.nb_edge.assign(ig.n, {});
  for (int v = 0; v < ig.n; ++v) ig.nb_edge[v].assign(ig.nb[v].size(), -1);
  for (int e = 0; e < gr.n_edges; ++e) {
    const int a = ig.edges[e].first, b = ig.edges[e].second;
    const int pa = (int)(std::find(ig.nb[a].begin(), ig.nb[a].end(), b) - ig.nb[a].begin());
    const int pb = (int)(std::find(ig.nb[b].begin(), ig.nb[b].end(), a) - ig.nb[b].begin());
    ig.nb_edge[a][pa] = e;
    ig.nb_edge[b][pb] = e;
  }
  ig.colour.assign(gr.n_edges, -1);
  if (gr.colour) {
    for (int e = 0; e < gr.n_edges; ++e) {
      if (gr.colour[e] < 0) return GPEPS_EINVAL;
      ig.colour[e] = gr.colour[e];
    }
  } else {
    // greedy first-fit over edges sorted by (smaller label, larger label)
    std::vector<int> order(gr.n_edges);
    for (int e = 0; e < gr.n_edges; ++e) order[e] = e;
    std::sort(order.begin(), order.end(), [&](int x, int y) {
      auto kx = std::make_pair(std::min(ig.edges[x].first, ig.edges[x].second),
                               std::max(ig.edges[x].first, ig.edges[x].second));
      auto ky = std::make_pair(std::min(ig.edges[y].first, ig.edges[y].second),
                               std::max(ig.edges[y].first, ig.edges[y].second));
      return kx < ky;
    });
    std::vector<unsigned> used(ig.n, 0u);  // colour bitmask per vertex
    for (int e : order) {
      const int a = ig.edges[e].first, b = ig.edges[e].second;
      const unsigned taken = used[a] | used[b];
      int c = 0;
      while (taken & (1u << c)) ++c;
      ig.colour[e] = c;
      used[a] |= 1u << c;
      used[b] |= 1u << c;
    }
  }
  // every class must be a matching
  std::vector<std::vector<int>> touched(ig.n);
  for (int e = 0; e < gr.n_edges; ++e) {
    for (int v : {ig.edges[e].first, ig.edges[e].second}) {
      for (int c : touched[v])
        if (c == ig.colour[e]) return GPEPS_EINVAL;
      touched[v].push_back(ig.colour[e]);
    }
  }
  return GPEPS_OK;
}

SideDesc side_desc(const gpeps_handle* h, int inst, int v, int nbr) {
  const InstGraph& ig = h->g[inst];
  const int D = h->D;
  const int d = (int)ig.nb[v].size();
  const int p = (int)(std::find(ig.nb[v].begin(), ig.nb[v].end(), nbr) - ig.nb[v].begin());
  auto stride = [&](int q) { return (int32_t)ipow(D, d - 1 - q); };
  SideDesc sd{};
  const int gsite = h->inst_site0[inst] + v;
  sd.off = h->site_off[gsite];
  sd.site = gsite;
  sd.str_s = (int32_t)ipow(D, d);
  sd.str_k = stride(p);
  sd.rows = (int32_t)ipow(D, d - 1);
  std::vector<int> others;
  for (int q = 0; q < d; ++q)
    if (q != p) others.push_back(q);
  const int e0 = h->inst_edge0[inst];
  sd.lam_o1 = sd.lam_o2 = -1;
  sd.str_o1 = sd.str_o2 = 0;
  sd.n2 = 1;
  if (others.size() == 2) {
    sd.str_o1 = stride(others[0]);
    sd.lam_o1 = (e0 + ig.nb_edge[v][others[0]]) * D;
    sd.str_o2 = stride(others[1]);
    sd.lam_o2 = (e0 + ig.nb_edge[v][others[1]]) * D;
    sd.n2 = D;
  } else if (others.size() == 1) {
    sd.str_o2 = stride(others[0]);
    sd.lam_o2 = (e0 + ig.nb_edge[v][others[0]]) * D;
    sd.n2 = D;
  }
  return sd;
}

struct PhaseEvents {
  cudaEvent_t ev[4];
};

// CTAs per SM of the layered bond launch (schedule 4 runs its layers, outside
// gpeps_step, on the work queue with two CTAs per SM where they fit)
int layered_per_sm(const gpeps_handle* h) {
  switch (h->schedule) {
    case 2: return 2;
    case 3: return 4;
    case 4:
    case 5:
    case 6: return bond_footprint_global(h->D, h->elt).smem <= bond_share_smem(2) ? 2 : 1;
    default: return 1;
  }
}

// CTAs per SM of the fused step launch
int step_per_sm(const gpeps_handle* h) {
  const size_t sm = step_footprint(h->D, h->elt, h->tensor).smem;
  if (h->schedule == 6 && sm <= bond_share_smem(4) && (!h->tensor || 4 * tc_cols(h->D) <= 512)) return 4;
  if (h->schedule >= 5 && sm <= bond_share_smem(3)) return 3;
  return sm <= bond_share_smem(2) ? 2 : 1;
}

template <typename T>
int fused_step_impl(gpeps_handle* h) {
  GP_CUDA(Launch<T>::step(h->at<StepTask>(h->w_tasks), (int)h->tasks.size(), h->at<unsigned int>(h->w_queue),
                          h->at<int>(h->w_done), h->gamma(), h->lam(), h->pending(), h->flags(), h->sweeps(),
                          h->cycles(), h->D, h->jp, h->stream, h->n_sms, h->d_work + h->w_bond_scratch,
                          h->bond_slot, step_per_sm(h), h->tensor));
  h->bonds_since_reset += (int64_t)h->tasks.size();
  return GPEPS_OK;
}

template <typename T>
int layer_impl(gpeps_handle* h, int c, PhaseEvents* pe = nullptr, void* vsave = nullptr) {
  ColourPlan& cp = h->colours[c];
  const int nt = (int)cp.tiles.size(), nbd = (int)cp.bonds.size();
  if (nbd == 0) return GPEPS_OK;
  const TileDesc* tiles = h->at<TileDesc>(cp.w_tiles);
  const BondDesc* bonds = h->at<BondDesc>(cp.w_bonds);
  void* partials = h->d_work + h->w_partials;
  void* Y = h->d_work + h->w_Y;
  double* theta_a = h->at<double>(h->w_theta_a);
  if (pe) GP_CUDA(cudaEventRecord(pe->ev[0], h->stream));
  if (h->tensor)
    GP_CUDA(Launch<T>::gram_tc(bonds, nbd, h->gamma(), h->lam(), h->pending(), partials, h->flags(), h->D,
                               h->stream));
  else
    GP_CUDA(Launch<T>::gram(tiles, nt, bonds, h->gamma(), h->lam(), h->pending(), partials, h->D, h->stream));
  if (pe) GP_CUDA(cudaEventRecord(pe->ev[1], h->stream));
  GP_CUDA(Launch<T>::bond(bonds, nbd, partials, h->gamma(), h->lam(), h->pending(), Y, theta_a, h->flags(),
                          h->sweeps(), h->cycles(), vsave, h->D, h->jp, h->stream,
                          h->schedule ? h->at<unsigned int>(h->w_queue) : nullptr, h->n_sms,
                          h->d_work + h->w_bond_scratch, layered_per_sm(h)));
  if (pe) GP_CUDA(cudaEventRecord(pe->ev[2], h->stream));
  if (h->tensor)
    GP_CUDA(Launch<T>::update_tc(bonds, nbd, h->gamma(), h->lam(), Y, theta_a, h->flags(), h->D, h->stream));
  else
    GP_CUDA(Launch<T>::update(tiles, nt, bonds, h->gamma(), h->lam(), Y, theta_a, h->D, h->stream));
  if (pe) GP_CUDA(cudaEventRecord(pe->ev[3], h->stream));
  h->bonds_since_reset += nbd;
  return GPEPS_OK;
}

int layer(gpeps_handle* h, int c, PhaseEvents* pe = nullptr, void* vsave = nullptr) {
  return h->dtype == GPEPS_C128 ? layer_impl<double>(h, c, pe, vsave) : layer_impl<float>(h, c, pe, vsave);
}

int kick_impl(gpeps_handle* h, const double* theta, int per_qubit, double scale = 1.0) {
  const int n = (int)h->total_sites;
  cudaError_t e = h->dtype == GPEPS_C128
                      ? Launch<double>::kick(h->pending(), theta, h->at<int32_t>(h->w_site_inst), n, per_qubit,
                                             h->stream, scale)
                      : Launch<float>::kick(h->pending(), theta, h->at<int32_t>(h->w_site_inst), n, per_qubit,
                                            h->stream, scale);
  if (e != cudaSuccess) return cuda_fail(e, "kick");
  return GPEPS_OK;
}

int readout_impl(gpeps_handle* h) {
  const int n = (int)h->total_sites;
  cudaError_t e =
      h->dtype == GPEPS_C128
          ? Launch<double>::readout(h->at<SiteDesc>(h->w_sites), n, h->gamma(), h->lam(), h->pending(), h->z(),
                                    h->D, h->stream)
          : Launch<float>::readout(h->at<SiteDesc>(h->w_sites), n, h->gamma(), h->lam(), h->pending(), h->z(),
                                   h->D, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "readout");
  e = launch_mean(h->z(), h->at<int32_t>(h->w_inst_site0), h->n_inst, h->mean(), h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mean");
  return GPEPS_OK;
}

int one_step(gpeps_handle* h, const double* theta, int per_qubit) {
  int st = kick_impl(h, theta, per_qubit);
  if (st) return st;
  if (h->schedule >= 4) {
    st = h->dtype == GPEPS_C128 ? fused_step_impl<double>(h) : fused_step_impl<float>(h);
    if (st) return st;
  } else {
    for (int c = 0; c < (int)h->colours.size(); ++c) {
      st = layer(h, c);
      if (st) return st;
    }
  }
  return readout_impl(h);
}

void drop_graph(gpeps_handle* h) {
  if (h->step_exec) cudaGraphExecDestroy(h->step_exec);
  h->step_exec = nullptr;
  h->step_theta = nullptr;
  h->step_per_qubit = -1;
}

}  // namespace

extern "C" {

int gpeps_create(const gpeps_graph* graphs, int32_t n_instances, int32_t D, int32_t dtype, void* stream,
                 gpeps_handle** out) {
  if (!out || !graphs || n_instances < 1) return GPEPS_EINVAL;
  *out = nullptr;
  if (dtype != GPEPS_C128 && dtype != GPEPS_MIXED_C64) return GPEPS_EINVAL;
  // complex128 (the unsquared bond SVD) reaches D = 128; the mixed path's squared
  // eigensolver keeps its n x n matrices and pair lists within D = 64
  if (D < 1 || D > (dtype == GPEPS_C128 ? kMaxDc128 : kMaxD)) return GPEPS_EINVAL;
  gpeps_handle* h = new (std::nothrow) gpeps_handle();
  if (!h) return GPEPS_ENOMEM;
  h->D = D;
  h->dtype = dtype;
  h->n_inst = n_instances;
  h->elt = dtype == GPEPS_C128 ? 16 : 8;
  h->stream = static_cast<cudaStream_t>(stream);
  h->g.resize(n_instances);
  for (int k = 0; k < n_instances; ++k) {
    const int st = validate_and_colour(graphs[k], h->g[k]);
    if (st) {
      delete h;
      return st;
    }
  }
  // sites, offsets
  h->inst_site0.assign(n_instances + 1, 0);
  h->inst_edge0.assign(n_instances + 1, 0);
  for (int k = 0; k < n_instances; ++k) {
    h->inst_site0[k + 1] = h->inst_site0[k] + h->g[k].n;
    h->inst_edge0[k + 1] = h->inst_edge0[k] + (int)h->g[k].edges.size();
  }
  h->total_sites = h->inst_site0[n_instances];
  h->total_edges = h->inst_edge0[n_instances];
  h->site_off.resize(h->total_sites);
  h->site_inst.resize(h->total_sites);
  h->sites.resize(h->total_sites);
  int64_t off = 0;
  for (int k = 0; k < n_instances; ++k) {
    for (int v = 0; v < h->g[k].n; ++v) {
      const int gs = h->inst_site0[k] + v;
      const int d = (int)h->g[k].nb[v].size();
      h->site_off[gs] = off;
      h->site_inst[gs] = k;
      SiteDesc sd{};
      sd.off = off;
      sd.deg = d;
      for (int q = 0; q < 3; ++q) sd.lam[q] = q < d ? (h->inst_edge0[k] + h->g[k].nb_edge[v][q]) * D : -1;
      h->sites[gs] = sd;
      off += 2 * ipow(D, d);
    }
  }
  h->n_gamma = off;
  // colour plans
  int ncol = 0;
  for (auto& ig : h->g)
    for (int c : ig.colour) ncol = std::max(ncol, c + 1);
  h->colours.resize(ncol);
  for (int c = 0; c < ncol; ++c) {
    ColourPlan& cp = h->colours[c];
    for (int k = 0; k < n_instances; ++k) {
      const InstGraph& ig = h->g[k];
      for (int e = 0; e < (int)ig.edges.size(); ++e) {
        if (ig.colour[e] != c) continue;
        int u = ig.edges[e].first, v = ig.edges[e].second;
        const int du = (int)ig.nb[u].size(), dv = (int)ig.nb[v].size();
        // end a: more legs (ties: smaller label); end b carries the eigenproblem
        int a = u, b = v;
        if (dv > du || (dv == du && v < u)) std::swap(a, b);
        BondDesc bd{};
        bd.a = side_desc(h, k, a, b);
        bd.b = side_desc(h, k, b, a);
        bd.lam_e = (h->inst_edge0[k] + e) * D;
        cp.bonds.push_back(bd);
      }
    }
    // largest bond eigenproblems (and larger ends) first: the last CTAs of a launch,
    // and the tail of the persistent work queue, are the cheap ones
    std::stable_sort(cp.bonds.begin(), cp.bonds.end(), [](const BondDesc& x, const BondDesc& y) {
      if (x.b.rows != y.b.rows) return x.b.rows > y.b.rows;
      return x.a.rows > y.a.rows;
    });
    for (int bi = 0; bi < (int)cp.bonds.size(); ++bi) {
      BondDesc& bd = cp.bonds[bi];
      bd.part0 = cp.n_parts;
      const int tr = tile_rows(D, dtype == GPEPS_C128 ? 16 : 8);
      bd.n_parts = (bd.a.rows + tr - 1) / tr;
      for (int p = 0; p < bd.n_parts; ++p) {
        TileDesc t{};
        t.bond = bi;
        t.row0 = p * tr;
        t.nrows = std::min(tr, bd.a.rows - t.row0);
        t.part = cp.n_parts + p;
        cp.tiles.push_back(t);
      }
      cp.n_parts += bd.n_parts;
    }
    h->max_parts = std::max(h->max_parts, cp.n_parts);
    h->max_bonds = std::max(h->max_bonds, (int)cp.bonds.size());
  }
  // fused step: every bond of a step, colour by colour; a task waits for the
  // last earlier task on each of its sites.  Class 0 keeps its cost order; a
  // later class is ordered by its latest dependency (then cost), so that the
  // tasks taken first are those whose sites were freed first.
  {
    std::vector<int> last((size_t)h->total_sites, -1);
    for (auto& cp : h->colours) {
      std::vector<int> idx(cp.bonds.size());
      for (int i = 0; i < (int)idx.size(); ++i) idx[i] = i;
      auto dep = [&](int i) { return std::max(last[cp.bonds[i].a.site], last[cp.bonds[i].b.site]); };
      std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return dep(x) < dep(y); });
      const int c = (int)(&cp - h->colours.data());
      std::vector<std::pair<int, int>> touched;
      for (int i : idx) {
        StepTask t{};
        t.bd = cp.bonds[i];
        t.dep_a = last[t.bd.a.site];
        t.dep_b = last[t.bd.b.site];
        t.colour = c;
        touched.emplace_back(t.bd.a.site, (int)h->tasks.size());
        touched.emplace_back(t.bd.b.site, (int)h->tasks.size());
        h->tasks.push_back(t);
      }
      for (auto& pr : touched) last[pr.first] = pr.second;
    }
  }
  // Jacobi thresholds.  Mixed: the FP64 sweeps on the squared bond matrix stop at
  // |a_pq| <= max(tol sqrt(a_pp a_qq), floor_rel * trace), a decade below the
  // ~1e-7 * trace rounding that rho inherits from its FP32 inputs (resolving that
  // rho further only fits noise).  Complex128: the one-sided sweeps on the bond
  // core stop at |b_p^H b_q| <= max(tol |b_p| |b_q|, floor_rel * ||M||_F^2): tol
  // at the rounding of a dot product of 2D terms (~2D eps), and a floor far
  // below it so that Schmidt values down to ~1e-10 of the largest are resolved
  // against each other (a floor at eps left lambda ~1e-8 off by 2e-8; at 1e-20
  // lambda stays within 7e-11 of the oracle, at 1e-24 within 7e-13 for a
  // quarter more FP64 work)
  h->jp.tol = dtype == GPEPS_C128 ? 1e-14 : 1e-9;
  h->jp.floor_rel = dtype == GPEPS_C128 ? 1e-20 : 1e-8;
  h->jp.tol32 = 1e-6;
  h->jp.floor32 = 2e-7;
  h->jp.ev_cut = 0.0;
  h->jp.max_sweeps = 40;
  h->jp.max_sweeps32 = 20;
  h->jp.level_ratio = 1e-5;
  h->jp.levels = 4;
  // beyond D = 64 one task of the fused step (Gram pass over 16384 rows, bond SVD,
  // update pass) takes about a second on its SM: its dependants may wait longer
  h->jp.wait_cycles = kWaitCycles * (D > kMaxD ? 16 : 1);
  h->jp.gate_sign = 1;
  // layouts
  size_t s = 0;
  h->s_lam = s;
  s = align256(s + (size_t)h->total_edges * D * sizeof(double));
  h->s_gamma = s;
  s = align256(s + (size_t)h->n_gamma * h->elt);
  h->state_bytes = std::max<size_t>(s, 256);
  size_t w = 0;
  auto carve = [&](size_t bytes) {
    const size_t o = w;
    w = align256(w + std::max<size_t>(bytes, 1));
    return o;
  };
  h->w_pending = carve(h->total_sites * sizeof(double));
  h->w_flags = carve(sizeof(int) * 4);
  h->w_sweeps = carve(kWorkCounters * sizeof(unsigned long long));
  h->w_cycles = carve(kCounters * sizeof(unsigned long long));
  h->w_queue = carve(sizeof(unsigned int));
  h->w_z = carve(h->total_sites * sizeof(double));
  h->w_mean = carve(n_instances * sizeof(double));
  h->w_sites = carve(h->total_sites * sizeof(SiteDesc));
  h->w_inst_site0 = carve((n_instances + 1) * sizeof(int32_t));
  h->w_site_inst = carve(h->total_sites * sizeof(int32_t));
  h->w_site_off = carve(h->total_sites * sizeof(int64_t));
  for (auto& cp : h->colours) {
    cp.w_bonds = carve(cp.bonds.size() * sizeof(BondDesc));
    cp.w_tiles = carve(cp.tiles.size() * sizeof(TileDesc));
  }
  h->w_partials = carve((size_t)h->max_parts * 2 * D * D * h->elt);
  h->w_Y = carve((size_t)h->max_bonds * 2 * D * D * h->elt);
  h->w_theta_a = carve((size_t)h->max_bonds * sizeof(double));
  // n x n bond matrices outside shared memory (a CTA indexes its slot by
  // blockIdx.x): beyond the shared-memory limit one slot per bond of the largest
  // class; otherwise slots for the two-CTAs-per-SM schedule only
  // (slots of the fused step are larger: they also hold the Gram sums and Y)
  h->bond_slot = std::max(bond_footprint_global(D, h->elt).slot, step_footprint(D, h->elt).slot);
  h->bond_slots = bond_footprint(D, kBondSmemMax, h->elt).slot ? h->max_bonds : std::min(h->max_bonds, 4 * kMaxSms);
  h->bond_slots = std::max(h->bond_slots, std::min((int)h->tasks.size(), 2 * kMaxSms));
  // four fused-step CTAs per SM where their shared memory fits (schedule 6)
  if (h->elt == 8 && step_footprint(D, h->elt, false).smem <= bond_share_smem(4))
    h->bond_slots = std::max(h->bond_slots, std::min((int)h->tasks.size(), 4 * kMaxSms));
  h->w_bond_scratch = carve((size_t)h->bond_slots * h->bond_slot);
  h->w_tasks = carve(h->tasks.size() * sizeof(StepTask));
  h->w_done = carve(h->tasks.size() * sizeof(int));
  h->work_bytes = w;
  *out = h;
  return GPEPS_OK;
}

int gpeps_query_workspace(const gpeps_handle* h, size_t* state_bytes, size_t* work_bytes) {
  if (!h || !state_bytes || !work_bytes) return GPEPS_EINVAL;
  *state_bytes = h->state_bytes;
  *work_bytes = h->work_bytes;
  return GPEPS_OK;
}

int gpeps_bind(gpeps_handle* h, void* d_state, void* d_work) {
  if (!h || !d_state || !d_work) return GPEPS_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_state) & 255) || (reinterpret_cast<uintptr_t>(d_work) & 255))
    return GPEPS_EINVAL;
  drop_graph(h);
  h->d_state = static_cast<char*>(d_state);
  h->d_work = static_cast<char*>(d_work);
  GP_CUDA(h->dtype == GPEPS_C128 ? Launch<double>::init() : Launch<float>::init());
  {
    int dev = 0;
    GP_CUDA(cudaGetDevice(&dev));
    GP_CUDA(cudaDeviceGetAttribute(&h->n_sms, cudaDevAttrMultiProcessorCount, dev));
    int optin = 0;
    GP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if ((size_t)optin < kSmemOptin) return GPEPS_EINVAL;  // not an sm_100-class device
  }
  auto up = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(h->d_work + off, src, bytes, cudaMemcpyHostToDevice, h->stream);
  };
  GP_CUDA(up(h->w_sites, h->sites.data(), h->sites.size() * sizeof(SiteDesc)));
  GP_CUDA(up(h->w_inst_site0, h->inst_site0.data(), h->inst_site0.size() * sizeof(int32_t)));
  GP_CUDA(up(h->w_site_inst, h->site_inst.data(), h->site_inst.size() * sizeof(int32_t)));
  GP_CUDA(up(h->w_site_off, h->site_off.data(), h->site_off.size() * sizeof(int64_t)));
  for (auto& cp : h->colours) {
    GP_CUDA(up(cp.w_bonds, cp.bonds.data(), cp.bonds.size() * sizeof(BondDesc)));
    GP_CUDA(up(cp.w_tiles, cp.tiles.data(), cp.tiles.size() * sizeof(TileDesc)));
  }
  GP_CUDA(up(h->w_tasks, h->tasks.data(), h->tasks.size() * sizeof(StepTask)));
  GP_CUDA(cudaMemsetAsync(h->d_work + h->w_flags, 0, sizeof(int) * 4, h->stream));
  GP_CUDA(cudaMemsetAsync(h->d_work + h->w_sweeps, 0, kWorkCounters * sizeof(unsigned long long), h->stream));
  GP_CUDA(cudaMemsetAsync(h->d_work + h->w_pending, 0, h->total_sites * sizeof(double), h->stream));
  // host vectors are pageable: the copies above have been staged when they return
  h->bound = true;
  return GPEPS_OK;
}

int gpeps_reset(gpeps_handle* h) {
  if (!h || !h->bound) return GPEPS_EINVAL;
  const int64_t* so = h->at<int64_t>(h->w_site_off);
  cudaError_t e = h->dtype == GPEPS_C128
                      ? Launch<double>::reset(h->gamma(), h->lam(), h->n_gamma, h->total_edges, h->D, so,
                                              (int)h->total_sites, h->pending(), h->stream)
                      : Launch<float>::reset(h->gamma(), h->lam(), h->n_gamma, h->total_edges, h->D, so,
                                             (int)h->total_sites, h->pending(), h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reset");
  GP_CUDA(cudaMemsetAsync(h->d_work + h->w_flags, 0, sizeof(int) * 4, h->stream));
  GP_CUDA(cudaMemsetAsync(h->d_work + h->w_sweeps, 0, kWorkCounters * sizeof(unsigned long long), h->stream));
  GP_CUDA(cudaMemsetAsync(h->d_work + h->w_cycles, 0, kCounters * sizeof(unsigned long long), h->stream));
  h->bonds_since_reset = 0;
  return GPEPS_OK;
}

int gpeps_kick(gpeps_handle* h, const double* theta, int32_t per_qubit) {
  if (!h || !h->bound || !theta) return GPEPS_EINVAL;
  return kick_impl(h, theta, per_qubit ? 1 : 0);
}

int gpeps_zz_layer(gpeps_handle* h, int32_t colour) {
  if (!h || !h->bound) return GPEPS_EINVAL;
  if (colour < 0 || colour >= (int)h->colours.size()) return GPEPS_EINVAL;
  return layer(h, colour);
}

int gpeps_zz_layer_profiled(gpeps_handle* h, int32_t colour, float* ms) {
  if (!h || !h->bound || !ms) return GPEPS_EINVAL;
  if (colour < 0 || colour >= (int)h->colours.size()) return GPEPS_EINVAL;
  PhaseEvents pe{};
  for (int i = 0; i < 4; ++i) GP_CUDA(cudaEventCreate(&pe.ev[i]));
  int st = layer(h, colour, &pe);
  cudaError_t e = cudaEventSynchronize(pe.ev[3]);
  for (int i = 0; i < 3 && st == GPEPS_OK && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&ms[i], pe.ev[i], pe.ev[i + 1]);
  for (int i = 0; i < 4; ++i) cudaEventDestroy(pe.ev[i]);
  if (st) return st;
  if (e != cudaSuccess) return cuda_fail(e, "gpeps_zz_layer_profiled");
  return GPEPS_OK;
}

int gpeps_step_profiled(gpeps_handle* h, const double* theta, int32_t per_qubit, float* ms) {
  if (!h || !h->bound || !theta || !ms) return GPEPS_EINVAL;
  cudaEvent_t ev[4];
  for (int i = 0; i < 4; ++i) GP_CUDA(cudaEventCreate(&ev[i]));
  auto body = [&]() -> int {
    GP_CUDA(cudaEventRecord(ev[0], h->stream));
    int st = kick_impl(h, theta, per_qubit ? 1 : 0);
    if (st) return st;
    GP_CUDA(cudaEventRecord(ev[1], h->stream));
    if (h->schedule >= 4) {
      st = h->dtype == GPEPS_C128 ? fused_step_impl<double>(h) : fused_step_impl<float>(h);
    } else {
      for (int c = 0; c < (int)h->colours.size() && !st; ++c) st = layer(h, c);
    }
    if (st) return st;
    GP_CUDA(cudaEventRecord(ev[2], h->stream));
    st = readout_impl(h);
    if (st) return st;
    GP_CUDA(cudaEventRecord(ev[3], h->stream));
    GP_CUDA(cudaEventSynchronize(ev[3]));
    for (int i = 0; i < 3; ++i) GP_CUDA(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
    return GPEPS_OK;
  };
  const int st = body();
  for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  return st;
}

int gpeps_set_schedule(gpeps_handle* h, int32_t schedule) {
  if (!h || schedule < 0 || schedule > 6) return GPEPS_EINVAL;
  if (schedule == 5 && (!h->bound || step_footprint(h->D, h->elt, h->tensor).smem > bond_share_smem(3) ||
                        std::min(3 * h->n_sms, (int)h->tasks.size()) > h->bond_slots))
    return GPEPS_EINVAL;
  if (schedule == 6 && (!h->bound || h->dtype != GPEPS_MIXED_C64 ||
                        step_footprint(h->D, h->elt, h->tensor).smem > bond_share_smem(4) ||
                        (h->tensor && 4 * tc_cols(h->D) > 512) ||
                        std::min(4 * h->n_sms, (int)h->tasks.size()) > h->bond_slots))
    return GPEPS_EINVAL;
  if (schedule >= 4) {
    // fused step: shared memory of one CTA (alone or two per SM) and a slot per CTA
    if (!h->bound) return GPEPS_EINVAL;
    const BondFootprint fp = step_footprint(h->D, h->elt, h->tensor);
    if (fp.smem > kBondSmemMax || fp.slot > h->bond_slot) return GPEPS_EINVAL;
    if (std::min(2 * h->n_sms, (int)h->tasks.size()) > h->bond_slots) return GPEPS_EINVAL;
    // its layers (gpeps_zz_layer) run two CTAs per SM where they fit
    const bool pair = bond_footprint_global(h->D, h->elt).smem <= bond_share_smem(2);
    if (pair && std::min(2 * h->n_sms, h->max_bonds) > h->bond_slots) return GPEPS_EINVAL;
  }
  if (schedule == 2 || schedule == 3) {
    // k CTAs per SM: shared memory of the FP32 level and a slot per CTA
    const int k = schedule == 3 ? 4 : 2;
    if (!h->bound || bond_footprint_global(h->D, h->elt).smem > bond_share_smem(k)) return GPEPS_EINVAL;
    if (std::min(k * h->n_sms, h->max_bonds) > h->bond_slots) return GPEPS_EINVAL;
  }
  h->schedule = schedule;
  drop_graph(h);
  return GPEPS_OK;
}

int gpeps_set_tensor_cores(gpeps_handle* h, int32_t on) {
  if (!h) return GPEPS_EINVAL;
  if (!on) {
    h->tensor = false;
    drop_graph(h);
    return GPEPS_OK;
  }
  if (h->dtype != GPEPS_MIXED_C64 || !tc_supported(h->D)) return GPEPS_EINVAL;
  // the fused schedule in use must still fit with the staged tensor-core operands
  if (h->schedule == 5 && step_footprint(h->D, h->elt, true).smem > bond_share_smem(3)) return GPEPS_EINVAL;
  if (h->schedule == 4 && step_footprint(h->D, h->elt, true).smem > kBondSmemMax) return GPEPS_EINVAL;
  // four CTAs per SM: shared memory of the staged operands, and four times the TMEM columns
  if (h->schedule == 6 && (step_footprint(h->D, h->elt, true).smem > bond_share_smem(4) || 4 * tc_cols(h->D) > 512))
    return GPEPS_EINVAL;
  h->tensor = true;
  drop_graph(h);
  return GPEPS_OK;
}

int gpeps_n_colours(const gpeps_handle* h, int32_t* n_colours) {
  if (!h || !n_colours) return GPEPS_EINVAL;
  *n_colours = (int32_t)h->colours.size();
  return GPEPS_OK;
}

int gpeps_expect_z(gpeps_handle* h, double* d_z, double* d_mean) {
  if (!h || !h->bound) return GPEPS_EINVAL;
  const int st = readout_impl(h);
  if (st) return st;
  if (d_z)
    GP_CUDA(cudaMemcpyAsync(d_z, h->z(), h->total_sites * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  if (d_mean)
    GP_CUDA(cudaMemcpyAsync(d_mean, h->mean(), h->n_inst * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  return GPEPS_OK;
}

int gpeps_inverse_steps(gpeps_handle* h, int32_t n_steps, const double* theta, int32_t per_qubit) {
  if (!h || !h->bound || !theta || n_steps < 0) return GPEPS_EINVAL;
  // U(theta) = ZZ K(theta), so U^dagger(theta) = K(-theta) ZZ^dagger: the colour
  // classes with the conjugate gate, in the reverse order of a forward step,
  // then the kick by -theta (pending, fused into the next bond or the readout)
  const int saved = h->jp.gate_sign;
  h->jp.gate_sign = -1;
  int st = GPEPS_OK;
  for (int t = 0; t < n_steps && !st; ++t) {
    for (int c = (int)h->colours.size() - 1; c >= 0 && !st; --c) st = layer(h, c);
    if (!st) st = kick_impl(h, theta, per_qubit ? 1 : 0, -1.0);
  }
  h->jp.gate_sign = saved;
  return st;
}

int gpeps_step(gpeps_handle* h, int32_t n_steps, const double* theta, int32_t per_qubit,
               double* d_mean_per_step) {
  if (!h || !h->bound || !theta || n_steps < 0) return GPEPS_EINVAL;
  per_qubit = per_qubit ? 1 : 0;
  const int64_t nbonds_step = [&] {
    int64_t s = 0;
    for (auto& cp : h->colours) s += (int64_t)cp.bonds.size();
    return s;
  }();
  const bool use_graph = h->stream != nullptr;
  if (use_graph && (h->step_exec == nullptr || h->step_theta != theta || h->step_per_qubit != per_qubit)) {
    drop_graph(h);
    GP_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    const int64_t saved = h->bonds_since_reset;
    const int st = one_step(h, theta, per_qubit);
    h->bonds_since_reset = saved;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->stream, &graph);
    if (st) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture");
    const cudaError_t ei = cudaGraphInstantiate(&h->step_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      h->step_exec = nullptr;
      return cuda_fail(ei, "cudaGraphInstantiate");
    }
    h->step_theta = theta;
    h->step_per_qubit = per_qubit;
  }
  for (int t = 0; t < n_steps; ++t) {
    if (use_graph) {
      GP_CUDA(cudaGraphLaunch(h->step_exec, h->stream));
      h->bonds_since_reset += nbonds_step;
    } else {
      const int st = one_step(h, theta, per_qubit);
      if (st) return st;
    }
    if (d_mean_per_step)
      GP_CUDA(cudaMemcpyAsync(d_mean_per_step + (int64_t)t * h->n_inst, h->mean(), h->n_inst * sizeof(double),
                              cudaMemcpyDeviceToDevice, h->stream));
  }
  return GPEPS_OK;
}

int gpeps_status(gpeps_handle* h, int32_t* flags) {
  if (!h || !h->bound || !flags) return GPEPS_EINVAL;
  GP_CUDA(cudaStreamSynchronize(h->stream));
  int f = 0;
  GP_CUDA(cudaMemcpy(&f, h->flags(), sizeof(int), cudaMemcpyDeviceToHost));
  *flags = f;
  return GPEPS_OK;
}

int gpeps_lambda(gpeps_handle* h, int32_t instance, int32_t edge, double* out) {
  if (!h || !h->bound || !out || instance < 0 || instance >= h->n_inst) return GPEPS_EINVAL;
  if (edge < 0 || edge >= (int)h->g[instance].edges.size()) return GPEPS_EINVAL;
  GP_CUDA(cudaStreamSynchronize(h->stream));
  GP_CUDA(cudaMemcpy(out, h->lam() + (int64_t)(h->inst_edge0[instance] + edge) * h->D, h->D * sizeof(double),
                     cudaMemcpyDeviceToHost));
  std::sort(out, out + h->D, [](double x, double y) { return x > y; });
  return GPEPS_OK;
}

int gpeps_site_layout(const gpeps_handle* h, int32_t instance, int32_t site, int64_t* byte_offset, int32_t* deg,
                      int32_t* neighbours) {
  if (!h || instance < 0 || instance >= h->n_inst) return GPEPS_EINVAL;
  if (site < 0 || site >= h->g[instance].n) return GPEPS_EINVAL;
  const int gs = h->inst_site0[instance] + site;
  const auto& nb = h->g[instance].nb[site];
  if (byte_offset) *byte_offset = (int64_t)h->s_gamma + h->site_off[gs] * (int64_t)h->elt;
  if (deg) *deg = (int32_t)nb.size();
  if (neighbours)
    for (int q = 0; q < 3; ++q) neighbours[q] = q < (int)nb.size() ? nb[q] : -1;
  return GPEPS_OK;
}

int gpeps_lambda_layout(const gpeps_handle* h, int32_t instance, int32_t edge, int64_t* byte_offset) {
  if (!h || !byte_offset || instance < 0 || instance >= h->n_inst) return GPEPS_EINVAL;
  if (edge < 0 || edge >= (int)h->g[instance].edges.size()) return GPEPS_EINVAL;
  *byte_offset = (int64_t)h->s_lam + (int64_t)(h->inst_edge0[instance] + edge) * h->D * (int64_t)sizeof(double);
  return GPEPS_OK;
}

int gpeps_sizes(const gpeps_handle* h, int64_t* total_qubits, int64_t* total_edges) {
  if (!h) return GPEPS_EINVAL;
  if (total_qubits) *total_qubits = h->total_sites;
  if (total_edges) *total_edges = h->total_edges;
  return GPEPS_OK;
}

int gpeps_sweeps(gpeps_handle* h, int64_t* sweeps64, int64_t* sweeps32, int64_t* total_bonds) {
  if (!h || !h->bound) return GPEPS_EINVAL;
  GP_CUDA(cudaStreamSynchronize(h->stream));
  unsigned long long s[2] = {0, 0};
  GP_CUDA(cudaMemcpy(s, h->sweeps(), sizeof(s), cudaMemcpyDeviceToHost));
  if (sweeps64) *sweeps64 = (int64_t)s[0];
  if (sweeps32) *sweeps32 = (int64_t)s[1];
  if (total_bonds) *total_bonds = h->bonds_since_reset;
  return GPEPS_OK;
}

int gpeps_jacobi_work(gpeps_handle* h, int64_t* work) {
  if (!h || !h->bound || !work) return GPEPS_EINVAL;
  GP_CUDA(cudaStreamSynchronize(h->stream));
  unsigned long long w[kWorkCounters];
  GP_CUDA(cudaMemcpy(w, h->sweeps(), sizeof(w), cudaMemcpyDeviceToHost));
  for (int i = 0; i < 4; ++i) work[i] = (int64_t)w[4 + i];
  work[4] = (int64_t)w[3];
  return GPEPS_OK;
}

int gpeps_bond_phase_cycles(gpeps_handle* h, int64_t* cycles) {
  if (!h || !h->bound || !cycles) return GPEPS_EINVAL;
  GP_CUDA(cudaStreamSynchronize(h->stream));
  unsigned long long c[kCounters];
  GP_CUDA(cudaMemcpy(c, h->cycles(), sizeof(c), cudaMemcpyDeviceToHost));
  for (int i = 0; i < kCounters; ++i) cycles[i] = (int64_t)c[i];
  return GPEPS_OK;
}

int gpeps_set_jacobi(gpeps_handle* h, double tol, double floor_rel, double tol32, double floor32,
                     int32_t max_sweeps, int32_t max_sweeps32) {
  if (!h) return GPEPS_EINVAL;
  if (!(tol > 0.0) || !(floor_rel > 0.0) || !(tol32 > 0.0) || !(floor32 > 0.0)) return GPEPS_EINVAL;
  if (max_sweeps < 1 || max_sweeps > 200 || max_sweeps32 < 0 || max_sweeps32 > 200) return GPEPS_EINVAL;
  h->jp.tol = tol;
  h->jp.floor_rel = floor_rel;
  h->jp.tol32 = tol32;
  h->jp.floor32 = floor32;
  h->jp.max_sweeps = max_sweeps;
  h->jp.max_sweeps32 = max_sweeps32;
  drop_graph(h);  // the captured step holds the old parameters
  return GPEPS_OK;
}

int gpeps_set_wait_limit(gpeps_handle* h, int64_t cycles) {
  if (!h || cycles < 0) return GPEPS_EINVAL;
  h->jp.wait_cycles = cycles;
  drop_graph(h);
  return GPEPS_OK;
}

int gpeps_set_levels(gpeps_handle* h, double level_ratio, int32_t levels) {
  if (!h) return GPEPS_EINVAL;
  if (!(level_ratio > 0.0 && level_ratio < 1.0) || levels < 0 || levels > kMaxExtraLevels) return GPEPS_EINVAL;
  h->jp.level_ratio = level_ratio;
  h->jp.levels = levels;
  drop_graph(h);
  return GPEPS_OK;
}

namespace {

struct GradLayout {
  size_t ckpt = 0, snaps = 0, adj = 0, partG = 0, partY = 0, Gbar = 0, Ybuf = 0, vsave = 0, vslot = 0, total = 0;
  int n_ckpt = 0, n_snap = 0;
};

GradLayout grad_layout(const gpeps_handle* h, int n_steps, int k) {
  GradLayout L;
  const size_t sb = h->state_bytes;
  const int nc = (int)h->colours.size();
  L.n_ckpt = (n_steps + k - 1) / k;
  L.n_snap = nc * k;
  size_t o = 0;
  L.ckpt = o;
  o += (size_t)L.n_ckpt * sb;
  L.snaps = o;
  o += (size_t)L.n_snap * sb;
  L.adj = o;
  o += sb;
  const size_t blk = (size_t)2 * h->D * h->D * 16;
  L.partG = o;
  o += align256((size_t)h->max_parts * blk);
  L.partY = o;
  o += align256((size_t)h->max_parts * blk);
  L.Gbar = o;
  o += align256((size_t)h->max_bonds * blk);
  L.Ybuf = o;
  o += align256((size_t)h->max_bonds * blk);
  // forward eigenvectors of every bond of every layer of a segment (2D x 2D + 2D complex per bond)
  const size_t nm = 2 * (size_t)h->D;
  L.vslot = align256((size_t)h->max_bonds * (nm * nm + nm) * 16);
  L.vsave = o;
  o += (size_t)L.n_snap * L.vslot;
  L.total = o;
  return L;
}

int grad_check(const gpeps_handle* h, int n_steps, int k) {
  if (!h || h->dtype != GPEPS_C128 || h->D > kMaxGradD || n_steps < 0 || k < 1) return GPEPS_EINVAL;
  return GPEPS_OK;
}

JacobiParams grad_jacobi(const gpeps_handle* h) {
  JacobiParams jp = h->jp;
  jp.ev_cut = 1e-14;  // Schmidt values <= 1e-7 of the largest are zero in both directions
  return jp;
}

}  // namespace

int gpeps_query_grad_workspace(const gpeps_handle* h, int32_t n_steps, int32_t ckpt_every, size_t* bytes) {
  if (!bytes) return GPEPS_EINVAL;
  const int st = grad_check(h, n_steps, ckpt_every);
  if (st) return st;
  *bytes = grad_layout(h, n_steps, ckpt_every).total;
  return GPEPS_OK;
}

int gpeps_grad(gpeps_handle* h, const double* theta, int32_t n_steps, int32_t ckpt_every, const double* dL_dz,
               double* z_out, double* dtheta, void* d_grad_work, size_t grad_work_bytes) {
  int st = grad_check(h, n_steps, ckpt_every);
  if (st) return st;
  if (!h->bound || !theta || !d_grad_work || (reinterpret_cast<uintptr_t>(d_grad_work) & 255)) return GPEPS_EINVAL;
  if (dL_dz && !dtheta) return GPEPS_EINVAL;
  const int k = ckpt_every;
  const GradLayout L = grad_layout(h, n_steps, k);
  if (grad_work_bytes < L.total) return GPEPS_EINVAL;
  char* gw = static_cast<char*>(d_grad_work);
  const size_t sb = h->state_bytes;
  const int nc = (int)h->colours.size();
  const int n_sites = (int)h->total_sites;
  const SiteDesc* sites = h->at<SiteDesc>(h->w_sites);
  cudaStream_t s = h->stream;
  const JacobiParams jp = grad_jacobi(h);
  const JacobiParams saved_jp = h->jp;
  GP_CUDA(Adjoint::init());
  GP_CUDA(Launch<double>::init());
  auto state_of = [&](char* base) { return std::make_pair(static_cast<void*>(base + h->s_gamma),
                                                          reinterpret_cast<double*>(base + h->s_lam)); };
  auto copy_state = [&](char* dst, const char* src) -> cudaError_t {
    return cudaMemcpyAsync(dst, src, sb, cudaMemcpyDeviceToDevice, s);
  };
  // forward layers of the gradient path: pending kicks are zero (kicks applied explicitly)
  auto fwd_layer = [&](int c, void* vsave) -> int {
    h->jp = jp;
    const int r = layer(h, c, nullptr, vsave);
    h->jp = saved_jp;
    return r;
  };
  // ---- forward with checkpoints
  st = gpeps_reset(h);
  if (st) return st;
  for (int t = 0; t < n_steps; ++t) {
    if (t % k == 0) GP_CUDA(copy_state(gw + L.ckpt + (size_t)(t / k) * sb, h->d_state));
    GP_CUDA(Adjoint::apply_kick(sites, n_sites, h->gamma(), theta, h->D, s));
    for (int c = 0; c < nc; ++c) {
      st = fwd_layer(c, nullptr);
      if (st) return st;
    }
  }
  st = readout_impl(h);
  if (st) return st;
  if (z_out) GP_CUDA(cudaMemcpyAsync(z_out, h->z(), n_sites * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (!dL_dz) return GPEPS_OK;
  // ---- reverse
  char* adj = gw + L.adj;
  GP_CUDA(cudaMemsetAsync(adj, 0, sb, s));
  GP_CUDA(cudaMemsetAsync(dtheta, 0, n_sites * sizeof(double), s));
  {
    auto cur = state_of(h->d_state);
    auto ad = state_of(adj);
    GP_CUDA(Adjoint::readout(sites, n_sites, cur.first, cur.second, dL_dz, ad.first, ad.second, h->D, s));
  }
  for (int seg = L.n_ckpt - 1; seg >= 0; --seg) {
    const int t0 = seg * k, t1 = std::min(n_steps, t0 + k);
    GP_CUDA(copy_state(h->d_state, gw + L.ckpt + (size_t)seg * sb));
    for (int t = t0; t < t1; ++t) {
      GP_CUDA(Adjoint::apply_kick(sites, n_sites, h->gamma(), theta, h->D, s));
      for (int c = 0; c < nc; ++c) {
        const size_t slot = (size_t)((t - t0) * nc + c);
        GP_CUDA(copy_state(gw + L.snaps + slot * sb, h->d_state));
        st = fwd_layer(c, gw + L.vsave + slot * L.vslot);
        if (st) return st;
      }
    }
    for (int t = t1 - 1; t >= t0; --t) {
      for (int c = nc - 1; c >= 0; --c) {
        ColourPlan& cp = h->colours[c];
        char* snap = gw + L.snaps + (size_t)((t - t0) * nc + c) * sb;
        auto in = state_of(snap);
        auto ad = state_of(adj);
        GP_CUDA(Adjoint::layer(h->at<TileDesc>(cp.w_tiles), (int)cp.tiles.size(), h->at<BondDesc>(cp.w_bonds),
                               (int)cp.bonds.size(), in.first, in.second, ad.first, ad.second, gw + L.partG,
                               gw + L.partY, gw + L.Gbar, gw + L.Ybuf,
                               gw + L.vsave + (size_t)((t - t0) * nc + c) * L.vslot, h->D, jp, s));
      }
      char* snap0 = gw + L.snaps + (size_t)((t - t0) * nc) * sb;
      auto post = state_of(snap0);
      auto ad = state_of(adj);
      GP_CUDA(Adjoint::kick(sites, n_sites, post.first, ad.first, theta, dtheta, h->D, s));
    }
  }
  return GPEPS_OK;
}

namespace {

// ---------------------------------------------------------------- BP regauging
void bp_plan(gpeps_handle* h) {
  if (!h->he0.empty()) return;
  const int D = h->D;
  h->he0.assign(h->total_sites + 1, 0);
  for (int64_t gs = 0; gs < h->total_sites; ++gs) h->he0[gs + 1] = h->he0[gs] + h->sites[gs].deg;
  h->n_half = h->he0[h->total_sites];
  for (int want = 3; want >= 1; --want) {  // the costly messages and sites first
    for (int k = 0; k < h->n_inst; ++k) {
      const InstGraph& ig = h->g[k];
      for (int v = 0; v < ig.n; ++v) {
        const int gs = h->inst_site0[k] + v;
        const SiteDesc& sd = h->sites[gs];
        if (sd.deg != want) continue;
        for (int p = 0; p < sd.deg; ++p) {
          BpMsgTask t{};
          t.off = sd.off;
          t.deg = sd.deg;
          t.leg = p;
          t.out = h->he0[gs] + p;
          for (int q = 0; q < 3; ++q) {
            t.in[q] = -1;
            t.lam[q] = q < sd.deg ? sd.lam[q] : 0;
            if (q < sd.deg) {
              const int nbr = ig.nb[v][q];
              const int back = (int)(std::find(ig.nb[nbr].begin(), ig.nb[nbr].end(), v) - ig.nb[nbr].begin());
              t.in[q] = h->he0[h->inst_site0[k] + nbr] + back;
            }
          }
          h->bp_msgs.push_back(t);
        }
        BpSiteTask st{};
        st.off = sd.off;
        st.deg = sd.deg;
        st.h0 = h->he0[gs];
        h->bp_sites.push_back(st);
      }
    }
  }
  for (int k = 0; k < h->n_inst; ++k) {
    const InstGraph& ig = h->g[k];
    for (int e = 0; e < (int)ig.edges.size(); ++e) {
      const int u = ig.edges[e].first, v = ig.edges[e].second;
      const int pu = (int)(std::find(ig.nb[u].begin(), ig.nb[u].end(), v) - ig.nb[u].begin());
      const int pv = (int)(std::find(ig.nb[v].begin(), ig.nb[v].end(), u) - ig.nb[v].begin());
      BpEdgeTask t{};
      t.hi = h->he0[h->inst_site0[k] + u] + pu;
      t.hj = h->he0[h->inst_site0[k] + v] + pv;
      t.lam = (h->inst_edge0[k] + e) * D;
      h->bp_edges.push_back(t);
    }
  }
}

struct BpLayout {
  size_t msg_a, msg_b, P, tasks, edges, sites, residual, scratch, total;
  int64_t slot_elems;  // complex elements (of the storage type for messages, FP64 for the gauge) per CTA slot
  int n_ctas;
};

// One message CTA per resident slot (occupancy of the message kernel at this D),
// so that the CTAs' scratch tensors stay in L2.  The launchers' shared-memory
// limits are raised first: the occupancy depends on them.
int bp_ctas(const gpeps_handle* h) {
  if (h->dtype == GPEPS_C128) BpLaunch<double>::init();
  else BpLaunch<float>::init();
  const int per_sm = h->dtype == GPEPS_C128 ? BpLaunch<double>::resident(h->D) : BpLaunch<float>::resident(h->D);
  return std::max(1, h->n_sms) * std::max(1, per_sm);
}

BpLayout bp_layout(const gpeps_handle* h, int max_iter) {
  BpLayout L{};
  const int D = h->D;
  const size_t msg = align256((size_t)h->n_half * D * D * sizeof(double2));
  int maxdeg = 0;
  for (const SiteDesc& sd : h->sites) maxdeg = std::max(maxdeg, (int)sd.deg);
  const int n = D + (D & 1);
  const int64_t site_elems = ipow(D, std::max(maxdeg, 1));  // one physical component of the largest site
  const size_t slot = std::max((size_t)site_elems * h->elt, (size_t)7 * n * n * sizeof(double2));
  L.slot_elems = (int64_t)(align256(slot) / 16);  // in units of 16 bytes
  L.n_ctas = bp_ctas(h);
  size_t o = 0;
  L.msg_a = o;
  o += msg;
  L.msg_b = o;
  o += msg;
  L.P = o;
  o += msg;
  L.tasks = o;
  o += align256(h->bp_msgs.size() * sizeof(BpMsgTask));
  L.edges = o;
  o += align256(h->bp_edges.size() * sizeof(BpEdgeTask));
  L.sites = o;
  o += align256(h->bp_sites.size() * sizeof(BpSiteTask));
  L.residual = o;
  o += align256((size_t)max_iter * sizeof(unsigned long long));
  L.scratch = o;
  o += (size_t)L.n_ctas * (size_t)L.slot_elems * 16;
  L.total = o;
  return L;
}

}  // namespace

int gpeps_query_bp_workspace(gpeps_handle* h, int32_t max_iter, size_t* bytes) {
  if (!h || !h->bound || !bytes || max_iter < 1 || h->D > kMaxD) return GPEPS_EINVAL;
  bp_plan(h);
  *bytes = bp_layout(h, max_iter).total;
  return GPEPS_OK;
}

int gpeps_bp_regauge(gpeps_handle* h, int32_t max_iter, double tol, void* d_bp_work, size_t bp_work_bytes,
                     int32_t* iterations, double* residual, float* phase_ms) {
  if (!h || !h->bound || max_iter < 1 || !(tol >= 0.0) || !d_bp_work || h->D > kMaxD) return GPEPS_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_bp_work) & 255) return GPEPS_EINVAL;
  bp_plan(h);
  const BpLayout L = bp_layout(h, max_iter);
  if (bp_work_bytes < L.total) return GPEPS_EINVAL;
  char* w = static_cast<char*>(d_bp_work);
  cudaStream_t s = h->stream;
  const int D = h->D;
  const bool c128 = h->dtype == GPEPS_C128;
  GP_CUDA(c128 ? BpLaunch<double>::init() : BpLaunch<float>::init());
  auto up = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(w + off, src, bytes, cudaMemcpyHostToDevice, s);
  };
  GP_CUDA(up(L.tasks, h->bp_msgs.data(), h->bp_msgs.size() * sizeof(BpMsgTask)));
  GP_CUDA(up(L.edges, h->bp_edges.data(), h->bp_edges.size() * sizeof(BpEdgeTask)));
  GP_CUDA(up(L.sites, h->bp_sites.data(), h->bp_sites.size() * sizeof(BpSiteTask)));
  GP_CUDA(cudaMemsetAsync(w + L.residual, 0, (size_t)max_iter * sizeof(unsigned long long), s));
  double2* cur = reinterpret_cast<double2*>(w + L.msg_a);
  double2* nxt = reinterpret_cast<double2*>(w + L.msg_b);
  GP_CUDA(c128 ? BpLaunch<double>::identity(cur, (int)h->n_half, D, s)
               : BpLaunch<float>::identity(cur, (int)h->n_half, D, s));
  const BpMsgTask* tasks = reinterpret_cast<const BpMsgTask*>(w + L.tasks);
  unsigned long long* res = reinterpret_cast<unsigned long long*>(w + L.residual);
  void* scratch = w + L.scratch;
  const int64_t slot_t = L.slot_elems * 16 / (int64_t)h->elt;  // the slot in storage-type complex elements
  int it = 0;
  double r = 0.0;
  // optional device times of the phases (CUDA events on the stream): messages, gauge, apply
  struct Events {
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
    ~Events() {
      for (auto& x : e)
        if (x) cudaEventDestroy(x);
    }
  } evs;
  cudaEvent_t* ev = evs.e;
  float msg_ms = 0.f;
  if (phase_ms)
    for (int k = 0; k < 4; ++k) GP_CUDA(cudaEventCreate(&ev[k]));
  while (it < max_iter) {
    if (phase_ms) GP_CUDA(cudaEventRecord(ev[0], s));
    cudaError_t e = c128 ? BpLaunch<double>::message(tasks, (int)h->bp_msgs.size(), h->gamma(), h->lam(), cur, nxt,
                                                    scratch, slot_t, D, res + it, h->flags(), L.n_ctas, s)
                         : BpLaunch<float>::message(tasks, (int)h->bp_msgs.size(), h->gamma(), h->lam(), cur, nxt,
                                                   scratch, slot_t, D, res + it, h->flags(), L.n_ctas, s,
                                                   h->tensor && D == 32);
    GP_CUDA(e);
    if (phase_ms) GP_CUDA(cudaEventRecord(ev[1], s));
    unsigned long long bits = 0;
    GP_CUDA(cudaMemcpyAsync(&bits, res + it, sizeof(bits), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (phase_ms) {
      float t = 0.f;
      GP_CUDA(cudaEventElapsedTime(&t, ev[0], ev[1]));
      msg_ms += t;
    }
    double2* t = cur;
    cur = nxt;
    nxt = t;
    ++it;
    std::memcpy(&r, &bits, sizeof(r));
    if (h->bp_msgs.empty() || r <= tol) break;
  }
  double2* P = reinterpret_cast<double2*>(w + L.P);
  if (phase_ms) GP_CUDA(cudaEventRecord(ev[1], s));
  {
    const BpEdgeTask* et = reinterpret_cast<const BpEdgeTask*>(w + L.edges);
    const int ne = (int)h->bp_edges.size();
    double2* sc = reinterpret_cast<double2*>(scratch);
    GP_CUDA(c128 ? BpLaunch<double>::gauge(et, ne, cur, h->lam(), P, sc, L.slot_elems, D, h->flags(), L.n_ctas, s)
                 : BpLaunch<float>::gauge(et, ne, cur, h->lam(), P, sc, L.slot_elems, D, h->flags(), L.n_ctas, s));
  }
  if (phase_ms) GP_CUDA(cudaEventRecord(ev[2], s));
  GP_CUDA(c128 ? BpLaunch<double>::apply(reinterpret_cast<const BpSiteTask*>(w + L.sites), (int)h->bp_sites.size(),
                                          h->gamma(), P, D, s)
               : BpLaunch<float>::apply(reinterpret_cast<const BpSiteTask*>(w + L.sites), (int)h->bp_sites.size(),
                                         h->gamma(), P, D, s));
  if (phase_ms) {
    GP_CUDA(cudaEventRecord(ev[3], s));
    GP_CUDA(cudaEventSynchronize(ev[3]));
    float tg = 0.f, ta = 0.f;
    GP_CUDA(cudaEventElapsedTime(&tg, ev[1], ev[2]));
    GP_CUDA(cudaEventElapsedTime(&ta, ev[2], ev[3]));
    phase_ms[0] = msg_ms;
    phase_ms[1] = tg;
    phase_ms[2] = ta;
  }
  if (iterations) *iterations = it;
  if (residual) *residual = r;
  return GPEPS_OK;
}

int gpeps_destroy(gpeps_handle* h) {
  if (!h) return GPEPS_EINVAL;
  drop_graph(h);
  delete h;
  return GPEPS_OK;
}

const char* gpeps_error_string(int status) {
  switch (status) {
    case GPEPS_OK: return "ok";
    case GPEPS_EINVAL: return "invalid argument";
    case GPEPS_ECUDA: return "CUDA runtime error";
    case GPEPS_ENOCONV: return "Jacobi eigensolver hit its sweep cap";
    case GPEPS_ENUMERIC: return "non-finite or vanishing bond spectrum";
    case GPEPS_ENOMEM: return "host allocation failed";
    default: return "unknown status";
  }
}

const char* gpeps_last_cuda_error(void) { return g_last_cuda.c_str(); }

}  // extern "C"
