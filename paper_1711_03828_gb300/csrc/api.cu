// api.cu -- the C ABI of libsoma (declared in include/soma.h).
//
// A soma_t owns the device state of one system:
//   positions   3 FP32 planes x|y|z of M floats (one allocation, planes
//               256-byte aligned), unwrapped, dL units;
//   n[2]        packed occupation grids (A | B<<16), double-buffered: the
//               sweep of step s counts into n[(s+1)&1] while omega holds the
//               fields of n[s&1];
//   omega       two planes (A, B) of the storage type (FP32/BF16/FP16);
//   counters    sweep counter (the Philox word w), accepted moves, sticky
//               error bits, the field kernel's arrival counter;
//   scratch     FP64 partial sums of the observables and S(q) reductions.
// A cycle is two launches (sweep, fields); soma_sweep replays them from a
// CUDA graph of GRAPH_CHUNK cycles when timing is off.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/soma.h"
#include "kernels.h"

using namespace soma;

namespace {

// Message of the last failing call on this thread: a fixed buffer, so that
// reporting an error allocates nothing either.
constexpr size_t ERR_LEN = 512;
thread_local char g_last_error[ERR_LEN] = "";

soma_status fail(soma_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
soma_status fail(soma_status st, const char* fmt, ...) {
  char buf[ERR_LEN];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  memcpy(g_last_error, buf, ERR_LEN);
  return st;
}

// Keeps the current message across cleanup calls that may report errors of
// their own (restored when the guard goes out of scope).
struct KeepError {
  char saved[ERR_LEN];
  KeepError() { memcpy(saved, g_last_error, ERR_LEN); }
  ~KeepError() { memcpy(g_last_error, saved, ERR_LEN); }
};

soma_status cuda_fail(cudaError_t e, const char* what) {
  // a failed call also leaves its error as the runtime's "last error"; clear
  // it so that the next launch check reports only its own failure
  (void)cudaGetLastError();
  return fail(e == cudaErrorMemoryAllocation ? SOMA_ENOMEM : SOMA_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define SOMA_CUDA(call)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

constexpr uint32_t GRAPH_CHUNK = 16;
constexpr uint64_t MAX_M = 1ull << 40;
// Supported position range |x|, |y|, |z| < 2^18 dL (exact cell fold).
constexpr uint64_t POS_LIMIT = 1ull << 18;

}  // namespace

struct soma_t {
  soma_system_desc desc;
  Geom g;
  double Re;        // R_e0 in dL
  double a64;       // maximal displacement in dL
  float a32;
  double K_b;
  double rho_cell;  // rho_0 dL^3
  double sigma;     // bond component standard deviation in dL
  int grid_dtype;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint64_t M = 0;
  uint64_t plane = 0;  // floats per position plane (padded)
  float* pos = nullptr;
  uint32_t* n[2] = {nullptr, nullptr};
  void* w[2] = {nullptr, nullptr};
  unsigned long long* d_counters = nullptr;  // [0] sweep, [1] accepted
  unsigned* d_err = nullptr;                 // [0] error bits, [1] arrival counter,
                                             // [2] range flag of soma_set_positions
  double* d_scratch = nullptr;
  float4* d_smc = nullptr;                   // smart Monte Carlo table, smc_planes * cells, SMC only
  uint32_t smc_planes = 0;                   // one float4 plane per type (A, B or n_t types)
  bool pos_invalid = false;                  // soma_set_positions was given positions out of range
  float* d_ext = nullptr;                    // external potential, 2 * cells (lazy)
  uint8_t* d_forbidden = nullptr;            // forbidden cells, cells bytes (lazy)
  bool has_ext = false, has_forbidden = false;
  uint64_t* d_seq = nullptr;                 // mixture: type sequence per architecture
  uint8_t* d_arch = nullptr;                 // mixture: architecture per chain
  // molecular architectures of Sec. 3.2.1 (types in d_seq, molecules in d_arch)
  bool has_topo = false;
  uint64_t* d_topo_pmask = nullptr;          // 256 * 64 partner masks
  uint32_t* d_topo_ptab = nullptr;           // 256 * 64 per-particle table words
  double topo_bonds = 0.0;                   // bonds in the system
  uint8_t* d_topo_ttab = nullptr;            // 256 * 64 particle types
  uint8_t* d_topo_len = nullptr;             // 256 particle counts (the rest of N absent)
  uint64_t M_real = 0;                       // particles present (M less absent slots)
  uint32_t topo_max_type = 0;                // largest type of the current architectures
  // n_t particle types (0: the two types A, B of the packed grid)
  uint32_t n_types = 0;
  double chiN_types[TYPES_MAX * TYPES_MAX] = {};
  uint32_t* nt[2] = {nullptr, nullptr};      // count planes, n_types * cells each
  float* wt = nullptr;                       // field planes, n_types * cells
  int topo_grid = 1;
  double* d_out = nullptr;
  size_t scratch_doubles = 0;
  double* d_tw = nullptr;
  size_t tw_doubles = 0;
  SweepShape shape;
  uint64_t host_sweep = 0;
  uint64_t launches = 0;
  // chain sharding: 0 no exchange pending, 1 soma_shard_counts done, 2
  // soma_shard_sweep done (soma_shard_fields comes next in both cases)
  int shard_phase = 0;
  bool timing = false;
  struct EvPair { cudaEvent_t a, b; int kind; };
  std::vector<EvPair> ev_pending;
  std::vector<cudaEvent_t> ev_free;
  soma_timing t{};
  cudaGraphExec_t graph = nullptr;
  bool batched = false;  // advanced only through its soma_batch_t
  // learned proposal: FP32 master weights, BF16 copy, Adam moments, gradient
  float* mlp_w = nullptr;
  void* mlp_q = nullptr;
  float* mlp_m = nullptr;
  float* mlp_v = nullptr;
  float* mlp_g = nullptr;
  uint32_t train_step = 0;
  SweepShape plain_shape;  // uniform-move shape (training trajectories)

  float* x() { return pos; }
  float* y() { return pos + plane; }
  float* z() { return pos + 2 * plane; }
};

namespace {

soma_status validate(const soma_system_desc* d) {
  if (!d) return fail(SOMA_EINVAL, "desc is NULL");
  if (d->struct_size != sizeof(soma_system_desc))
    return fail(SOMA_EINVAL, "desc.struct_size %u != %zu", d->struct_size, sizeof(soma_system_desc));
  if (d->N < 1 || d->N > 256) return fail(SOMA_EINVAL, "N=%u outside 1..256", d->N);
  if (d->n_chains < 1) return fail(SOMA_EINVAL, "n_chains must be >= 1");
  if (d->n_chains > MAX_M / d->N) return fail(SOMA_EINVAL, "M = n_chains*N exceeds 2^40");
  if (!(d->f >= 0.0 && d->f <= 1.0)) return fail(SOMA_EINVAL, "f=%g outside [0,1]", d->f);
  uint64_t cells = 1;
  for (int k = 0; k < 3; ++k) {
    if (!(d->box_Re[k] > 0.0) || !std::isfinite(d->box_Re[k]))
      return fail(SOMA_EINVAL, "box_Re[%d]=%g must be > 0", k, d->box_Re[k]);
    if (d->grid[k] < 1 || d->grid[k] > 4096)
      return fail(SOMA_EINVAL, "grid[%d]=%u outside 1..4096", k, d->grid[k]);
    cells *= d->grid[k];
  }
  if (cells > 0x7FFFFFFFull) return fail(SOMA_EINVAL, "grid has %llu cells (max 2^31-1)",
                                         (unsigned long long)cells);
  const double dl0 = d->box_Re[0] / d->grid[0];
  for (int k = 1; k < 3; ++k) {
    const double dl = d->box_Re[k] / d->grid[k];
    if (std::fabs(dl - dl0) > 1e-9 * dl0)
      return fail(SOMA_EINVAL, "cells are not cubic: dL differs between axes 0 and %d", k);
  }
  if (!std::isfinite(d->chiN) || !std::isfinite(d->kappaN) || !std::isfinite(d->a_Re))
    return fail(SOMA_EINVAL, "chiN, kappaN and a_Re must be finite");
  if (d->move != SOMA_MOVE_UNIFORM && d->move != SOMA_MOVE_SMC && d->move != SOMA_MOVE_LEARNED)
    return fail(SOMA_EINVAL, "move=%d is not available", d->move);
  if (d->set_order != SOMA_SET_ORDER_RANDOM && d->set_order != SOMA_SET_ORDER_FIXED &&
      d->set_order != SOMA_ITERATION_MOLECULE)
    return fail(SOMA_EINVAL, "set_order=%d unknown", d->set_order);
  if (d->set_order == SOMA_ITERATION_MOLECULE && d->move != SOMA_MOVE_UNIFORM)
    return fail(SOMA_EINVAL, "the molecule-parallel iteration takes uniform moves");
  if (d->grid_dtype < 0 || d->grid_dtype > 2)
    return fail(SOMA_EINVAL, "grid_dtype=%d unknown", d->grid_dtype);
  if (d->flags & ~(SOMA_FLAG_NO_SORT | SOMA_FLAG_LEARNED_FP32 | SOMA_FLAG_LEARNED_UMMA))
    return fail(SOMA_EINVAL, "unknown flags 0x%x", d->flags);
  if (d->replica_id > 0xFFFFFFu) return fail(SOMA_EINVAL, "replica_id must be < 2^24");
  if (d->hamiltonian > 1) return fail(SOMA_EINVAL, "hamiltonian=%u unknown", d->hamiltonian);
  if (d->n_chains_total == 0 && d->chain_offset != 0)
    return fail(SOMA_EINVAL, "chain_offset=%llu needs n_chains_total (the whole system's chains)",
                (unsigned long long)d->chain_offset);
  if (d->n_chains_total != 0) {
    if (d->chain_offset > d->n_chains_total || d->n_chains > d->n_chains_total - d->chain_offset)
      return fail(SOMA_EINVAL, "chains [%llu, %llu) lie outside the %llu chains of the system",
                  (unsigned long long)d->chain_offset,
                  (unsigned long long)(d->chain_offset + d->n_chains),
                  (unsigned long long)d->n_chains_total);
    if (d->n_chains_total >= (1ull << 32) / d->N)
      return fail(SOMA_EINVAL, "a sharded system needs n_chains_total*N < 2^32");
  }
  return SOMA_OK;
}

void derive(soma_t* h) {
  const soma_system_desc& d = h->desc;
  h->Re = (double)d.grid[0] / d.box_Re[0];
  double a_Re = d.a_Re;
  if (!(a_Re > 0.0)) a_Re = (d.N > 1) ? 0.5 / std::sqrt((double)(d.N - 1)) : 0.5;
  h->a64 = a_Re * h->Re;
  h->a32 = (float)h->a64;
  h->K_b = (d.N > 1) ? 3.0 * (double)(d.N - 1) / (2.0 * h->Re * h->Re) : 0.0;
  h->sigma = (d.N > 1) ? h->Re / std::sqrt(3.0 * (double)(d.N - 1)) : 0.0;
  h->M = d.n_chains * d.N;
  h->M_real = h->M;
  const double cells = (double)d.grid[0] * (double)d.grid[1] * (double)d.grid[2];
  // rho_0 dL^3 of the whole system (a shard holds part of its particles)
  const uint64_t M_all = (d.n_chains_total ? d.n_chains_total : d.n_chains) * d.N;
  h->rho_cell = (double)M_all / cells;
  h->grid_dtype = d.grid_dtype;
  Geom& g = h->g;
  g.n_chains = d.n_chains;
  g.N = d.N;
  uint32_t NA = (uint32_t)std::floor(d.f * (double)d.N + 0.5);
  g.N_A = NA > d.N ? d.N : NA;
  g.nx = (int)d.grid[0];
  g.ny = (int)d.grid[1];
  g.nz = (int)d.grid[2];
  const uint32_t n3[3] = {d.grid[0], d.grid[1], d.grid[2]};
  for (int k = 0; k < 3; ++k) {  // cell fold constants (see fold_raw)
    const uint64_t n = n3[k];
    const uint64_t bias = n * ((POS_LIMIT + n - 1) / n);
    g.fold_m[k] = n > 1 ? (uint32_t)(((1ull << 32) + n - 1) / n) : 0u;
    g.fold_s[k] = n > 1 ? 1u : 0u;
    g.fold_b[k] = n > 1 ? (uint32_t)((bias - 0x4B400000ull) & 0xFFFFFFFFull) : 0u;
  }
  g.cells = (uint32_t)(d.grid[0] * d.grid[1] * d.grid[2]);
  g.key0 = (uint32_t)d.seed;
  g.key1 = (uint32_t)(d.seed >> 32);
  for (int r = 0; r < 10; ++r) {
    g.rk0[r] = g.key0 + (uint32_t)r * 0x9E3779B9u;
    g.rk1[r] = g.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  g.replica = d.replica_id;
  g.chain_base = d.n_chains_total ? d.chain_offset : 0;
  g.id_base = g.chain_base * d.N;
  g.particles = M_all;
}

size_t wbytes(int dtype) { return dtype == 0 ? 4 : 2; }

void release(soma_t* h) {
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (auto& p : h->ev_pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto e : h->ev_free) cudaEventDestroy(e);
  cudaFree(h->pos);
  cudaFree(h->n[0]);
  cudaFree(h->n[1]);
  cudaFree(h->w[0]);
  cudaFree(h->w[1]);
  cudaFree(h->d_counters);
  cudaFree(h->d_err);
  cudaFree(h->d_scratch);
  cudaFree(h->d_smc);
  cudaFree(h->d_ext);
  cudaFree(h->d_forbidden);
  cudaFree(h->d_seq);
  cudaFree(h->d_arch);
  cudaFree(h->d_topo_pmask);
  cudaFree(h->d_topo_ptab);
  cudaFree(h->d_topo_ttab);
  cudaFree(h->d_topo_len);
  cudaFree(h->nt[0]);
  cudaFree(h->nt[1]);
  cudaFree(h->wt);
  cudaFree(h->d_tw);
  cudaFree(h->mlp_w);
  cudaFree(h->mlp_q);
  cudaFree(h->mlp_m);
  cudaFree(h->mlp_v);
  cudaFree(h->mlp_g);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

FieldArgs field_args(soma_t* h, int after_sweep) {
  FieldArgs f;
  f.g = h->g;
  f.n0 = h->n[0];
  f.n1 = h->n[1];
  f.wA = h->w[0];
  f.wB = h->w[1];
  f.d_sweep = h->d_counters;
  f.err = h->d_err;
  f.inv_rho = (float)(1.0 / h->rho_cell);
  f.kappa0 = (float)(h->desc.kappaN / (double)h->desc.N);
  f.half_chi0 = (float)(0.5 * h->desc.chiN / (double)h->desc.N);
  f.after_sweep = after_sweep;
  f.hamiltonian = (int)h->desc.hamiltonian;
  f.ext = h->has_ext ? h->d_ext : nullptr;
  f.forbidden = h->has_forbidden ? h->d_forbidden : nullptr;
  return f;
}

SweepArgs sweep_args(soma_t* h) {
  SweepArgs s;
  s.g = h->g;
  s.x = h->x();
  s.y = h->y();
  s.z = h->z();
  s.wA = h->w[0];
  s.wB = h->w[1];
  s.n0 = h->n[0];
  s.n1 = h->n[1];
  s.acc = h->d_counters + 1;
  s.d_sweep = h->d_counters;
  s.a = h->a32;
  s.K_b = (float)h->K_b;
  s.G = h->shape.G;
  s.n_tiles = h->shape.n_tiles;
  s.full_tiles = h->g.n_chains / h->shape.G;
  s.last_rows = (uint32_t)(h->g.n_chains % h->shape.G) * h->g.N;
  s.set_order_random = h->desc.set_order == SOMA_SET_ORDER_RANDOM;
  const double A = h->a64 * h->a64 / 6.0;
  s.smc_A = (float)A;
  s.smc_s2A = (float)std::sqrt(2.0 * A);
  s.smc_inv4A = (float)(1.0 / (4.0 * A));
  s.learned_sigma0 = (float)(h->a64 / std::sqrt(3.0));
  s.smc_tab = h->d_smc;
  s.err = h->d_err;
  s.seq = h->d_seq;
  s.arch = h->d_seq ? h->d_arch : nullptr;
  return s;
}

cudaEvent_t take_event(soma_t* h) {
  if (!h->ev_free.empty()) {
    cudaEvent_t e = h->ev_free.back();
    h->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch one kernel (kind 0 sweep, 1 fields), bracketed by events if timing.
template <typename F>
soma_status timed(soma_t* h, int kind, F&& launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (h->timing) {
    a = take_event(h);
    b = take_event(h);
    SOMA_CUDA(cudaEventRecord(a, h->stream));
  }
  cudaError_t e = launch();
  if (e != cudaSuccess) return cuda_fail(e, kind == 0 ? "sweep kernel launch" : "field kernel launch");
  ++h->launches;
  if (kind == 0) ++h->t.sweep_launches; else ++h->t.field_launches;
  if (h->timing) {
    SOMA_CUDA(cudaEventRecord(b, h->stream));
    h->ev_pending.push_back({a, b, kind});
  }
  return SOMA_OK;
}

TopoArgs topo_args(soma_t* h, const SweepArgs& sa) {
  TopoArgs t;
  t.s = sa;
  t.pmask = h->d_topo_pmask;
  t.ptab = h->d_topo_ptab;
  t.mol_arch = h->d_arch;
  t.alen = h->d_topo_len;
  t.ttab = h->d_topo_ttab;
  t.wt = h->wt;
  t.nt0 = h->nt[0];
  t.nt1 = h->nt[1];
  return t;
}

TypesArgs types_args(soma_t* h, int after_sweep) {
  TypesArgs a;
  a.g = h->g;
  a.n0 = h->nt[0];
  a.n1 = h->nt[1];
  a.w = h->wt;
  a.d_sweep = h->d_counters;
  a.n_types = h->n_types;
  a.after_sweep = after_sweep;
  a.hamiltonian = (int)h->desc.hamiltonian;
  a.inv_rho = (float)(1.0 / h->rho_cell);
  a.inv_rho_f64 = 1.0 / h->rho_cell;
  a.kappa0 = (float)(h->desc.kappaN / (double)h->desc.N);
  for (int k = 0; k < TYPES_MAX * TYPES_MAX; ++k) {
    a.chiN[k] = h->chiN_types[k];
    a.chi0[k] = (float)(h->chiN_types[k] / (double)h->desc.N);
  }
  return a;
}

// the table of fields and field forces that smart Monte Carlo sweeps read,
// after every field update of such a system (A and B, or one plane per type)
cudaError_t launch_smc_table_of(soma_t* h) {
  if (!h->d_smc) return cudaSuccess;
  ++h->launches;
  if (h->n_types)
    return launch_smc_table_planes(h->g, h->wt, h->n_types, h->d_smc, h->sm_count, h->stream);
  return launch_smc_table(h->g, h->w[0], h->w[1], h->d_smc, h->grid_dtype, h->sm_count, h->stream);
}

// the field update of one cycle: the packed A | B grid or the type planes
cudaError_t launch_fields_any(soma_t* h, const FieldArgs& fa, const TypesArgs& ta) {
  cudaError_t e = h->n_types ? launch_fields_types(ta, h->d_err + 1, h->sm_count, h->stream)
                             : launch_fields(fa, h->d_err + 1, h->grid_dtype, h->sm_count, h->stream);
  if (e == cudaSuccess) e = launch_smc_table_of(h);
  return e;
}

cudaError_t launch_sweep_any(soma_t* h, const SweepArgs& sa) {
  const bool types = h->n_types != 0;
  if (h->has_topo && h->shape.molecule)
    return launch_molecule_topology(topo_args(h, sa), h->topo_grid, h->grid_dtype, h->stream,
                                    types);
  if (h->has_topo)
    return launch_sweep_topology(topo_args(h, sa), h->topo_grid, h->grid_dtype, h->shape.big,
                                 h->stream, types, h->desc.move == SOMA_MOVE_SMC);
  if (h->desc.move == SOMA_MOVE_LEARNED)
    return launch_sweep_learned(sa, h->shape, h->grid_dtype, h->mlp_q, h->stream);
  return launch_sweep_uniform(sa, h->shape, h->grid_dtype, h->stream);
}

soma_status one_cycle(soma_t* h) {
  const SweepArgs sa = sweep_args(h);
  soma_status st = timed(h, 0, [&] { return launch_sweep_any(h, sa); });
  if (st != SOMA_OK) return st;
  const FieldArgs fa = field_args(h, 1);
  const TypesArgs ta = types_args(h, 1);
  st = timed(h, 1, [&] { return launch_fields_any(h, fa, ta); });
  if (st != SOMA_OK) return st;
  ++h->host_sweep;
  return SOMA_OK;
}

soma_status build_graph(soma_t* h) {
  cudaGraph_t gr = nullptr;
  SOMA_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  const SweepArgs sa = sweep_args(h);
  const FieldArgs fa = field_args(h, 1);
  const TypesArgs ta = types_args(h, 1);
  cudaError_t e = cudaSuccess;
  for (uint32_t k = 0; k < GRAPH_CHUNK && e == cudaSuccess; ++k) {
    e = launch_sweep_any(h, sa);
    if (e == cudaSuccess) e = launch_fields_any(h, fa, ta);
  }
  cudaError_t e2 = cudaStreamEndCapture(h->stream, &gr);
  if (e != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return cuda_fail(e, "graph capture"); }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->graph, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) { h->graph = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
  return SOMA_OK;
}

soma_status check_sticky(soma_t* h) {
  unsigned err = 0;
  SOMA_CUDA(cudaMemcpy(&err, h->d_err, sizeof err, cudaMemcpyDeviceToHost));
  if (err & ERR_OVERFLOW) return fail(SOMA_EOVERFLOW, "a 16-bit occupation number reached 0xC000");
  if (err & ERR_TIMEOUT) return fail(SOMA_ETIMEOUT, "a bounded device wait gave up");
  return SOMA_OK;
}

soma_status sync(soma_t* h) {
  SOMA_CUDA(cudaStreamSynchronize(h->stream));
  return check_sticky(h);
}

soma_status update_fields(soma_t* h) {
  if (h->n_types && !h->has_topo)
    return fail(SOMA_ESTATE, "n_t types take the architecture path: call soma_set_topology");
  if (h->n_types) {   // count into the type planes nt[s&1], then the fields
    uint32_t* nn = h->nt[h->host_sweep & 1];
    SOMA_CUDA(cudaMemsetAsync(nn, 0, sizeof(uint32_t) * h->n_types * h->g.cells, h->stream));
    SOMA_CUDA(launch_histogram_types(h->g, h->x(), h->y(), h->z(), h->d_topo_ttab, h->d_arch, nn,
                                     h->sm_count, h->stream));
    SOMA_CUDA(launch_fields_types(types_args(h, 0), h->d_err + 1, h->sm_count, h->stream));
    h->launches += 2;
    SOMA_CUDA(launch_smc_table_of(h));
    return SOMA_OK;
  }
  // count into n[s&1] (cleared first), then omega from it
  uint32_t* nn = h->n[h->host_sweep & 1];
  SOMA_CUDA(cudaMemsetAsync(nn, 0, sizeof(uint32_t) * h->g.cells, h->stream));
  SOMA_CUDA(launch_histogram(h->g, h->x(), h->y(), h->z(), nn, h->sm_count, h->stream,
                             h->d_seq, h->d_seq ? h->d_arch : nullptr,
                             h->has_topo ? h->d_topo_len : nullptr));
  ++h->launches;
  const FieldArgs fa = field_args(h, 0);
  SOMA_CUDA(launch_fields(fa, h->d_err + 1, h->grid_dtype, h->sm_count, h->stream));
  ++h->launches;
  SOMA_CUDA(launch_smc_table_of(h));
  return SOMA_OK;
}

}  // namespace

namespace soma {
// Validation and geometry of a description for entry points that take no
// handle (same rules as soma_create).
soma_status describe(const soma_system_desc* d, Geom* g) {
  soma_status st = validate(d);
  if (st != SOMA_OK) return st;
  soma_t tmp;
  tmp.desc = *d;
  derive(&tmp);
  *g = tmp.g;
  return SOMA_OK;
}
soma_status report(soma_status st, const char* msg) { return fail(st, "%s", msg); }
soma_status report_cuda(cudaError_t e, const char* what) { return cuda_fail(e, what); }
}  // namespace soma

extern "C" {

int soma_abi_version(void) { return SOMA_ABI_VERSION; }

const char* soma_last_error(void) { return g_last_error; }

soma_status soma_create(const soma_system_desc* desc, soma_t** out) {
  if (!out) return fail(SOMA_EINVAL, "out is NULL");
  *out = nullptr;
  soma_status st = validate(desc);
  if (st != SOMA_OK) return st;
  soma_t* h = new (std::nothrow) soma_t();
  if (!h) return fail(SOMA_ENOMEM, "host allocation failed");
  h->desc = *desc;
  derive(h);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) { delete h; return cuda_fail(e, "device query"); }
  if (desc->stream) {
    h->stream = (cudaStream_t)desc->stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaStreamCreate"); }
    h->own_stream = true;
  }
  h->plane = (h->M + 63) & ~63ull;
  const size_t cells = h->g.cells;
  const size_t wb = wbytes(h->grid_dtype);
  h->scratch_doubles = (size_t)SQ_BLOCKS * 2 * SQ_MAX;
  if (h->scratch_doubles < 5 * (size_t)OBS_BLOCKS) h->scratch_doubles = 5 * (size_t)OBS_BLOCKS;
#define ALLOC(ptr, bytes)                                                   \
  do {                                                                      \
    e = cudaMalloc((void**)&(ptr), (bytes));                                \
    if (e != cudaSuccess) { release(h); return cuda_fail(e, "cudaMalloc " #ptr); } \
  } while (0)
  ALLOC(h->pos, sizeof(float) * 3 * h->plane);
  ALLOC(h->n[0], sizeof(uint32_t) * cells);
  ALLOC(h->n[1], sizeof(uint32_t) * cells);
  ALLOC(h->w[0], wb * cells);
  ALLOC(h->w[1], wb * cells);
  ALLOC(h->d_counters, sizeof(unsigned long long) * 2);
  ALLOC(h->d_err, sizeof(unsigned) * 3);
  ALLOC(h->d_scratch, sizeof(double) * (h->scratch_doubles + 64));
  ALLOC(h->mlp_w, sizeof(float) * SOMA_MLP_PARAMS);
  ALLOC(h->mlp_q, 2 * SOMA_MLP_PARAMS);
  ALLOC(h->mlp_m, sizeof(float) * SOMA_MLP_PARAMS);
  ALLOC(h->mlp_v, sizeof(float) * SOMA_MLP_PARAMS);
  ALLOC(h->mlp_g, sizeof(float) * SOMA_MLP_PARAMS);
  if (desc->move == SOMA_MOVE_SMC) {
    ALLOC(h->d_smc, sizeof(float4) * 2 * cells);
    h->smc_planes = 2;
  }
#undef ALLOC
  h->d_out = h->d_scratch + h->scratch_doubles;
  h->shape = sweep_shape(h->g.n_chains, h->g.N, h->sm_count, h->grid_dtype, desc->move,
                         (desc->flags & SOMA_FLAG_LEARNED_FP32) != 0,
                         (desc->flags & SOMA_FLAG_LEARNED_UMMA) != 0,
                         desc->set_order == SOMA_ITERATION_MOLECULE);
  h->plain_shape = sweep_shape(h->g.n_chains, h->g.N, h->sm_count, h->grid_dtype, SOMA_MOVE_UNIFORM);
#define CK(call) do { e = (call); if (e != cudaSuccess) { release(h); return cuda_fail(e, #call); } } while (0)
  CK(cudaMemsetAsync(h->n[0], 0, sizeof(uint32_t) * cells, h->stream));
  CK(cudaMemsetAsync(h->n[1], 0, sizeof(uint32_t) * cells, h->stream));
  CK(cudaMemsetAsync(h->d_counters, 0, sizeof(unsigned long long) * 2, h->stream));
  CK(cudaMemsetAsync(h->d_err, 0, sizeof(unsigned) * 3, h->stream));
  CK(cudaMemsetAsync(h->mlp_w, 0, sizeof(float) * SOMA_MLP_PARAMS, h->stream));
  CK(cudaMemsetAsync(h->mlp_q, 0, 2 * SOMA_MLP_PARAMS, h->stream));
  CK(cudaMemsetAsync(h->mlp_m, 0, sizeof(float) * SOMA_MLP_PARAMS, h->stream));
  CK(cudaMemsetAsync(h->mlp_v, 0, sizeof(float) * SOMA_MLP_PARAMS, h->stream));
  if ((desc->flags & SOMA_FLAG_NO_SORT) || h->g.n_chains >= (1ull << 32)) {
    CK(launch_init(h->g, h->x(), h->y(), h->z(), h->sigma, h->sm_count, h->stream));
    ++h->launches;
  } else {
    // draw the chains into a staging buffer, then store them in spatial order
    uint64_t n_pad = 1;
    while (n_pad < h->g.n_chains) n_pad <<= 1;
    float* stage = nullptr;
    uint64_t* keys = nullptr;
    e = cudaMallocAsync((void**)&stage, sizeof(float) * 3 * h->plane, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&keys, sizeof(uint64_t) * n_pad, h->stream);
    if (e == cudaSuccess)
      e = launch_init(h->g, stage, stage + h->plane, stage + 2 * h->plane, h->sigma, h->sm_count,
                      h->stream);
    if (e == cudaSuccess)
      e = launch_sort_chains(h->g, stage, h->plane, h->pos, h->plane, keys, n_pad, h->sm_count,
                             h->stream);
    if (stage) cudaFreeAsync(stage, h->stream);
    if (keys) cudaFreeAsync(keys, h->stream);
    if (e != cudaSuccess) { release(h); return cuda_fail(e, "initial configuration"); }
    h->launches += 3;
  }
#undef CK
  st = update_fields(h);
  if (st == SOMA_OK) st = sync(h);
  if (st != SOMA_OK) { KeepError keep; release(h); return st; }
  *out = h;
  return SOMA_OK;
}

soma_status soma_destroy(soma_t* h) {
  if (!h) return SOMA_OK;
  release(h);
  return SOMA_OK;
}

soma_status soma_sweep(soma_t* h, uint32_t n) {
  if (!h) return fail(SOMA_EINVAL, "handle is NULL");
  if (h->batched) return fail(SOMA_ESTATE, "this system belongs to a batch: use soma_batch_sweep");
  if (h->desc.n_chains_total)
    return fail(SOMA_ESTATE, "a shard exchanges counts every cycle: use soma_shard_sweep");
  if (h->pos_invalid) return fail(SOMA_ESTATE, "positions out of range: set valid positions first");
  if (h->n_types && !h->has_topo)
    return fail(SOMA_ESTATE, "n_t types take the architecture path: call soma_set_topology");
  uint32_t done = 0;
  if (!h->timing && n >= GRAPH_CHUNK) {
    if (!h->graph) {
      soma_status st = build_graph(h);
      if (st != SOMA_OK) return st;
    }
    while (n - done >= GRAPH_CHUNK) {
      SOMA_CUDA(cudaGraphLaunch(h->graph, h->stream));
      h->launches += (h->d_smc ? 3 : 2) * GRAPH_CHUNK;
      h->t.sweep_launches += GRAPH_CHUNK;
      h->t.field_launches += GRAPH_CHUNK;
      h->host_sweep += GRAPH_CHUNK;
      done += GRAPH_CHUNK;
    }
  }
  for (; done < n; ++done) {
    soma_status st = one_cycle(h);
    if (st != SOMA_OK) return st;
  }
  return SOMA_OK;
}

soma_status soma_update_fields(soma_t* h) {
  if (!h) return fail(SOMA_EINVAL, "handle is NULL");
  if (h->pos_invalid) return fail(SOMA_ESTATE, "positions out of range: set valid positions first");
  if (h->desc.n_chains_total)
    return fail(SOMA_ESTATE, "a shard's fields need every shard's counts: use soma_shard_counts");
  return update_fields(h);
}

namespace {
soma_status shard_check(soma_t* h, const void* buf, size_t cells) {
  if (!h || !buf) return fail(SOMA_EINVAL, "NULL argument");
  if (!h->desc.n_chains_total) return fail(SOMA_ESTATE, "not a shard (desc.n_chains_total is 0)");
  if (cells != h->g.cells) return fail(SOMA_EINVAL, "cells=%zu, the grid has %u", cells, h->g.cells);
  if (h->pos_invalid) return fail(SOMA_ESTATE, "positions out of range: set valid positions first");
  return SOMA_OK;
}
}  // namespace

soma_status soma_shard_counts(soma_t* h, uint32_t* counts, size_t cells) {
  soma_status st = shard_check(h, counts, cells);
  if (st != SOMA_OK) return st;
  if (h->shard_phase != 0) return fail(SOMA_ESTATE, "soma_shard_fields must come first");
  uint32_t* nn = h->n[h->host_sweep & 1];
  SOMA_CUDA(cudaMemsetAsync(nn, 0, sizeof(uint32_t) * cells, h->stream));
  SOMA_CUDA(launch_histogram(h->g, h->x(), h->y(), h->z(), nn, h->sm_count, h->stream,
                             h->d_seq, h->d_seq ? h->d_arch : nullptr,
                             h->has_topo ? h->d_topo_len : nullptr));
  ++h->launches;
  SOMA_CUDA(cudaMemcpyAsync(counts, nn, sizeof(uint32_t) * cells, cudaMemcpyDefault, h->stream));
  h->shard_phase = 1;
  return SOMA_OK;
}

soma_status soma_shard_sweep(soma_t* h, uint32_t* counts, size_t cells) {
  soma_status st = shard_check(h, counts, cells);
  if (st != SOMA_OK) return st;
  if (h->shard_phase != 0) return fail(SOMA_ESTATE, "soma_shard_fields must come first");
  const SweepArgs sa = sweep_args(h);
  st = timed(h, 0, [&] { return launch_sweep_any(h, sa); });
  if (st != SOMA_OK) return st;
  SOMA_CUDA(cudaMemcpyAsync(counts, h->n[(h->host_sweep + 1) & 1], sizeof(uint32_t) * cells,
                            cudaMemcpyDefault, h->stream));
  h->shard_phase = 2;
  return SOMA_OK;
}

soma_status soma_shard_fields(soma_t* h, const uint32_t* summed, size_t cells) {
  soma_status st = shard_check(h, summed, cells);
  if (st != SOMA_OK) return st;
  if (h->shard_phase == 0)
    return fail(SOMA_ESTATE, "soma_shard_counts or soma_shard_sweep must come first");
  const int after_sweep = h->shard_phase == 2;
  // the summed counts take the place of the shard's own in the buffer the
  // field kernel reads: n[(s+1)&1] after a sweep, n[s&1] otherwise
  uint32_t* nn = h->n[(h->host_sweep + (after_sweep ? 1 : 0)) & 1];
  SOMA_CUDA(cudaMemcpyAsync(nn, summed, sizeof(uint32_t) * cells, cudaMemcpyDefault, h->stream));
  const FieldArgs fa = field_args(h, after_sweep);
  st = timed(h, 1, [&] {
    cudaError_t e = launch_fields(fa, h->d_err + 1, h->grid_dtype, h->sm_count, h->stream);
    return e == cudaSuccess ? launch_smc_table_of(h) : e;
  });
  if (st != SOMA_OK) return st;
  if (after_sweep) ++h->host_sweep;
  h->shard_phase = 0;
  return SOMA_OK;
}

soma_status soma_sync(soma_t* h) {
  if (!h) return fail(SOMA_EINVAL, "handle is NULL");
  return sync(h);
}

void* soma_stream(soma_t* h) { return h ? (void*)h->stream : nullptr; }

soma_status soma_get_density(soma_t* h, uint32_t* dst, size_t n_cells, int dst_on_device) {
  if (!h || !dst) return fail(SOMA_EINVAL, "NULL argument");
  if (h->n_types) return fail(SOMA_EINVAL, "n_t types: use soma_get_type_counts");
  if (n_cells != h->g.cells) return fail(SOMA_EINVAL, "n_cells=%zu, grid has %u", n_cells, h->g.cells);
  const uint32_t* src = h->n[h->host_sweep & 1];
  SOMA_CUDA(cudaMemcpyAsync(dst, src, sizeof(uint32_t) * n_cells,
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            h->stream));
  return sync(h);
}

soma_status soma_get_fields(soma_t* h, float* dst, size_t n, int dst_on_device) {
  if (!h || !dst) return fail(SOMA_EINVAL, "NULL argument");
  if (h->n_types) return fail(SOMA_EINVAL, "n_t types: use soma_get_type_fields");
  const size_t cells = h->g.cells;
  if (n != 2 * cells) return fail(SOMA_EINVAL, "n=%zu, expected 2*cells=%zu", n, 2 * cells);
  if (h->grid_dtype == 0) {
    const cudaMemcpyKind k = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    SOMA_CUDA(cudaMemcpyAsync(dst, h->w[0], sizeof(float) * cells, k, h->stream));
    SOMA_CUDA(cudaMemcpyAsync(dst + cells, h->w[1], sizeof(float) * cells, k, h->stream));
    return sync(h);
  }
  float* tmp = dst;
  if (!dst_on_device) SOMA_CUDA(cudaMallocAsync((void**)&tmp, sizeof(float) * 2 * cells, h->stream));
  SOMA_CUDA(launch_convert_fields(h->w[0], h->grid_dtype, tmp, cells, h->stream));
  SOMA_CUDA(launch_convert_fields(h->w[1], h->grid_dtype, tmp + cells, cells, h->stream));
  h->launches += 2;
  if (!dst_on_device) {
    SOMA_CUDA(cudaMemcpyAsync(dst, tmp, sizeof(float) * 2 * cells, cudaMemcpyDeviceToHost, h->stream));
    SOMA_CUDA(cudaFreeAsync(tmp, h->stream));
  }
  return sync(h);
}

soma_status soma_get_positions(soma_t* h, float* dst, size_t n, int dst_on_device) {
  if (!h || !dst) return fail(SOMA_EINVAL, "NULL argument");
  if (n != 3 * h->M) return fail(SOMA_EINVAL, "n=%zu, expected 3*M=%llu", n, (unsigned long long)(3 * h->M));
  const cudaMemcpyKind k = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int d = 0; d < 3; ++d)
    SOMA_CUDA(cudaMemcpyAsync(dst + d * h->M, h->pos + d * h->plane, sizeof(float) * h->M, k, h->stream));
  return sync(h);
}

soma_status soma_set_positions(soma_t* h, const float* src, size_t n, int src_on_device) {
  if (!h || !src) return fail(SOMA_EINVAL, "NULL argument");
  if (n != 3 * h->M) return fail(SOMA_EINVAL, "n=%zu, expected 3*M=%llu", n, (unsigned long long)(3 * h->M));
  const cudaMemcpyKind k = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int d = 0; d < 3; ++d)
    SOMA_CUDA(cudaMemcpyAsync(h->pos + d * h->plane, src + d * h->M, sizeof(float) * h->M, k, h->stream));
  // every coordinate must lie in the supported range of the cell fold; the
  // check runs on the device copy, and a handle holding positions outside it
  // refuses to sweep until valid positions are set
  const float lim = (float)POS_LIMIT;
  unsigned flag = 0;
  SOMA_CUDA(cudaMemsetAsync(h->d_err + 2, 0, sizeof(unsigned), h->stream));
  for (int d = 0; d < 3; ++d)
    SOMA_CUDA(launch_range_check(h->pos + d * h->plane, h->M, lim, h->d_err + 2, h->sm_count, h->stream));
  SOMA_CUDA(cudaMemcpyAsync(&flag, h->d_err + 2, sizeof flag, cudaMemcpyDeviceToHost, h->stream));
  SOMA_CUDA(cudaStreamSynchronize(h->stream));
  h->launches += 3;
  h->pos_invalid = flag != 0;
  h->shard_phase = 0;
  if (flag)
    return fail(SOMA_EINVAL, "a position is not finite or has |x| >= 2^18 dL: set valid positions "
                             "before the next sweep");
  return SOMA_OK;
}

soma_status soma_set_external(soma_t* h, const float* ext, const uint8_t* forbidden,
                              int src_on_device) {
  if (!h) return fail(SOMA_EINVAL, "handle is NULL");
  if (forbidden && h->desc.move != SOMA_MOVE_UNIFORM)
    return fail(SOMA_EINVAL, "forbidden cells take uniform moves only");
  if (h->n_types && (ext || forbidden))
    return fail(SOMA_EINVAL, "external fields take the two types A, B");
  if (h->batched) return fail(SOMA_ESTATE, "a batch member has no external fields");
  const size_t cells = h->g.cells;
  const cudaMemcpyKind k = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e;
  if (ext) {
    if (!h->d_ext) {
      e = cudaMalloc((void**)&h->d_ext, sizeof(float) * 2 * cells);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc ext");
    }
    SOMA_CUDA(cudaMemcpyAsync(h->d_ext, ext, sizeof(float) * 2 * cells, k, h->stream));
  }
  if (forbidden) {
    if (!h->d_forbidden) {
      e = cudaMalloc((void**)&h->d_forbidden, cells);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc forbidden");
    }
    SOMA_CUDA(cudaMemcpyAsync(h->d_forbidden, forbidden, cells, k, h->stream));
  }
  h->has_ext = ext != nullptr;
  h->has_forbidden = forbidden != nullptr;
  // the captured cycle holds the old field-kernel arguments
  if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
  return sync(h);
}

namespace {
// Every slot of every molecule present: the density and particle count of the
// description (after architectures of fewer particles are replaced).
void restore_particles(soma_t* h) {
  soma_t tmp;
  tmp.desc = h->desc;
  derive(&tmp);
  h->rho_cell = tmp.rho_cell;
  h->g.particles = tmp.g.particles;
  h->M_real = h->M;
}
}  // namespace

soma_status soma_set_architectures(soma_t* h, const uint64_t* seq, uint32_t n_arch,
                                   const uint8_t* arch, int src_on_device) {
  if (!h) return fail(SOMA_EINVAL, "handle is NULL");
  if (h->batched) return fail(SOMA_ESTATE, "a batch member runs the diblock of its description");
  if (h->n_types) return fail(SOMA_ESTATE, "n_t types take architectures: call soma_set_types(h, 0, NULL) first");
  h->has_topo = false;
  h->topo_max_type = 0;
  restore_particles(h);
  if (!seq) {   // back to the diblock of the description
    cudaFree(h->d_seq);
    cudaFree(h->d_arch);
    h->d_seq = nullptr;
    h->d_arch = nullptr;
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    return SOMA_OK;
  }
  if (!arch || n_arch < 1 || n_arch > 256) return fail(SOMA_EINVAL, "need 1..256 architectures and arch");
  if (h->g.N > 64) return fail(SOMA_EINVAL, "mixtures take N <= 64");
  if (h->desc.move == SOMA_MOVE_LEARNED) return fail(SOMA_EINVAL, "mixtures take uniform or smart Monte Carlo moves");
  if (h->desc.move == SOMA_MOVE_UNIFORM && h->desc.set_order != SOMA_ITERATION_MOLECULE &&
      (h->g.N % 2 != 0 || h->shape.big))
    return fail(SOMA_EINVAL, "mixtures take even N (SET) or the molecule-parallel iteration");
  // every architecture index is checked on the host (it addresses seq)
  std::vector<uint8_t> a((size_t)h->g.n_chains);
  if (src_on_device)
    SOMA_CUDA(cudaMemcpy(a.data(), arch, a.size(), cudaMemcpyDeviceToHost));
  else
    std::memcpy(a.data(), arch, a.size());
  for (size_t k = 0; k < a.size(); ++k)
    if (a[k] >= n_arch) return fail(SOMA_EINVAL, "arch[%zu] = %u >= n_arch = %u", k, a[k], n_arch);
  if (h->desc.move == SOMA_MOVE_SMC) {
    // Smart Monte Carlo moves run on the architecture path: each linear
    // architecture written in the array layout of Sec. 3.2.1 (particle i of
    // type bit i of its sequence, bonded to i - 1 and i + 1).
    const uint32_t N = h->g.N;
    std::vector<uint64_t> sq(n_arch);
    SOMA_CUDA(cudaMemcpy(sq.data(), seq, sizeof(uint64_t) * n_arch,
                         src_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
    std::vector<uint32_t> words, start(n_arch);
    for (uint32_t k = 0; k < n_arch; ++k) {
      start[k] = (uint32_t)words.size();
      words.push_back(N);
      const size_t first = words.size();
      words.resize(first + N);
      for (uint32_t i = 0; i < N; ++i) {
        const uint32_t type = (uint32_t)((sq[k] >> i) & 1ull);
        if (N == 1) {
          words[first + i] = 0xFFFFFFu << 8 | type;   // a lone particle: no bonds
          continue;
        }
        words[first + i] = (uint32_t)words.size() << 8 | type;
        if (i > 0) words.push_back(0x7FFFFFFu << 5 | (i + 1 < N ? 0u : 1u));   // offset -1
        if (i + 1 < N) words.push_back(1u << 5 | 1u);                          // offset +1, last
      }
    }
    return soma_set_topology(h, words.data(), words.size(), start.data(), n_arch, a.data(), 0);
  }
  cudaError_t e;
  if (!h->d_seq) {
    e = cudaMalloc((void**)&h->d_seq, sizeof(uint64_t) * 256);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc seq");
  }
  if (!h->d_arch) {
    e = cudaMalloc((void**)&h->d_arch, a.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc arch");
  }
  SOMA_CUDA(cudaMemcpyAsync(h->d_seq, seq, sizeof(uint64_t) * n_arch,
                            src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  SOMA_CUDA(cudaMemcpyAsync(h->d_arch, a.data(), a.size(), cudaMemcpyHostToDevice, h->stream));
  if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
  return sync(h);
}

namespace {
// launch grid of the architecture sweep for the handle's iteration, move and types
void set_topo_grid(soma_t* h) {
  h->topo_grid = h->shape.molecule
                     ? molecule_topology_grid(h->g.N, h->grid_dtype, h->sm_count, h->g.n_chains)
                     : topology_grid(h->grid_dtype, h->shape.big, h->sm_count, h->shape.n_tiles,
                                     h->n_types != 0, h->desc.move == SOMA_MOVE_SMC);
}
}  // namespace

soma_status soma_set_topology(soma_t* h, const uint32_t* words, uint64_t n_words,
                              const uint32_t* start, uint32_t n_arch, const uint8_t* mol_arch,
                              int src_on_device) {
  if (!h) return fail(SOMA_EINVAL, "handle is NULL");
  if (h->batched) return fail(SOMA_ESTATE, "a batch member runs the diblock of its description");
  if (!words) return soma_set_architectures(h, nullptr, 0, nullptr, 0);
  if (!start || !mol_arch || n_arch < 1 || n_arch > 256 || n_words < 2 || n_words > (1ull << 24))
    return fail(SOMA_EINVAL, "need 1..256 architectures in 2..2^24 words, start and mol_arch");
  if (h->g.N > 64) return fail(SOMA_EINVAL, "architectures take N <= 64");
  if (h->desc.move == SOMA_MOVE_LEARNED)
    return fail(SOMA_EINVAL, "architectures take the uniform or smart Monte Carlo move");
  const cudaMemcpyKind k = src_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  std::vector<uint32_t> w((size_t)n_words), st(n_arch);
  std::vector<uint8_t> a((size_t)h->g.n_chains);
  SOMA_CUDA(cudaMemcpy(w.data(), words, sizeof(uint32_t) * w.size(), k));
  SOMA_CUDA(cudaMemcpy(st.data(), start, sizeof(uint32_t) * st.size(), k));
  SOMA_CUDA(cudaMemcpy(a.data(), mol_arch, a.size(), k));
  TopologyTables T;
  const std::string why = topology_tables(w.data(), n_words, st.data(), n_arch, h->g.N, &T,
                                          h->n_types ? h->n_types : 2u);
  if (!why.empty()) return fail(SOMA_EINVAL, "%s", why.c_str());
  double bonds = 0.0;
  uint64_t present = 0;
  for (size_t m = 0; m < a.size(); ++m) {
    if (a[m] >= n_arch) return fail(SOMA_EINVAL, "mol_arch[%zu] = %u >= n_arch = %u", m, a[m], n_arch);
    bonds += (double)T.bonds[a[m]];
    present += T.len[a[m]];
  }
  if (h->desc.n_chains_total && present != h->M)
    return fail(SOMA_EINVAL, "a shard takes architectures of N particles only (its density "
                             "counts the whole system)");
  cudaError_t e;
  if (!h->d_topo_pmask) {
    e = cudaMalloc((void**)&h->d_topo_pmask, sizeof(uint64_t) * 256 * 64);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_topo_ptab, sizeof(uint32_t) * 256 * 64);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_topo_ttab, 256 * 64);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_topo_len, 256);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc architecture tables");
  }
  if (!h->d_seq) {
    e = cudaMalloc((void**)&h->d_seq, sizeof(uint64_t) * 256);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc seq");
  }
  if (!h->d_arch) {
    e = cudaMalloc((void**)&h->d_arch, a.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc arch");
  }
  const cudaMemcpyKind up = cudaMemcpyHostToDevice;
  SOMA_CUDA(cudaMemcpyAsync(h->d_topo_pmask, T.pmask.data(), sizeof(uint64_t) * T.pmask.size(), up,
                            h->stream));
  SOMA_CUDA(cudaMemcpyAsync(h->d_topo_ptab, T.ptab.data(), sizeof(uint32_t) * T.ptab.size(), up,
                            h->stream));
  SOMA_CUDA(cudaMemcpyAsync(h->d_topo_ttab, T.ttab.data(), T.ttab.size(), up, h->stream));
  SOMA_CUDA(cudaMemcpyAsync(h->d_topo_len, T.len.data(), T.len.size(), up, h->stream));
  SOMA_CUDA(cudaMemcpyAsync(h->d_seq, T.seq.data(), sizeof(uint64_t) * n_arch, up, h->stream));
  SOMA_CUDA(cudaMemcpyAsync(h->d_arch, a.data(), a.size(), up, h->stream));
  soma_status s2 = sync(h);   // the host vectors are released on return
  if (s2 != SOMA_OK) return s2;
  h->topo_bonds = bonds;
  h->topo_max_type = T.max_type;
  // rho_0 dL^3 and the particle count follow the molecules' particles (a
  // shard holds molecules of N particles only and keeps the whole system's)
  h->M_real = present;
  if (!h->desc.n_chains_total) {
    h->g.particles = present;
    h->rho_cell = (double)present / (double)h->g.cells;
  }
  h->has_topo = true;
  set_topo_grid(h);
  if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
  return SOMA_OK;
}

soma_status soma_set_types(soma_t* h, uint32_t n_types, const double* chiN) {
  if (!h) return fail(SOMA_EINVAL, "handle is NULL");
  if (h->batched) return fail(SOMA_ESTATE, "a batch member has the two types A, B");
  if (h->desc.n_chains_total && n_types)
    return fail(SOMA_ESTATE, "a shard exchanges the packed A | B counts: n_t types are not sharded");
  if (n_types == 0) {   // back to the packed A | B grid
    if (h->topo_max_type > 1)
      return fail(SOMA_ESTATE, "the architectures use type %u: set two-type architectures first",
                  h->topo_max_type);
    cudaFree(h->nt[0]);
    cudaFree(h->nt[1]);
    cudaFree(h->wt);
    h->nt[0] = h->nt[1] = nullptr;
    h->wt = nullptr;
    h->n_types = 0;
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    if (h->has_topo) set_topo_grid(h);
    const soma_status st = update_fields(h);
    return st == SOMA_OK ? sync(h) : st;
  }
  if (n_types < 2 || n_types > (uint32_t)TYPES_MAX || !chiN)
    return fail(SOMA_EINVAL, "n_types=%u outside 2..%d, or chiN is NULL", n_types, TYPES_MAX);
  for (uint32_t i = 0; i < n_types; ++i)
    for (uint32_t j = 0; j < n_types; ++j) {
      const double a = chiN[i * n_types + j], b = chiN[j * n_types + i];
      if (!std::isfinite(a) || a != b || (i == j && a != 0.0))
        return fail(SOMA_EINVAL, "chiN must be finite and symmetric with a zero diagonal (%u, %u)",
                    i, j);
    }
  if (h->grid_dtype != 0) return fail(SOMA_EINVAL, "n_t types take FP32 fields");
  if (h->desc.move == SOMA_MOVE_LEARNED)
    return fail(SOMA_EINVAL, "n_t types take the uniform or smart Monte Carlo move");
  if (h->has_ext || h->has_forbidden) return fail(SOMA_EINVAL, "n_t types take no external fields");
  if (h->has_topo && h->topo_max_type >= n_types)
    return fail(SOMA_EINVAL, "the architectures use type %u >= n_types", h->topo_max_type);
  if (!h->has_topo && h->d_seq)
    return fail(SOMA_ESTATE, "a mixture of linear architectures has the two types A, B");
  const size_t bytes = sizeof(uint32_t) * n_types * h->g.cells;
  cudaFree(h->nt[0]);
  cudaFree(h->nt[1]);
  cudaFree(h->wt);
  h->nt[0] = h->nt[1] = nullptr;
  h->wt = nullptr;
  h->n_types = 0;
  cudaError_t e = cudaMalloc((void**)&h->nt[0], bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->nt[1], bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->wt, sizeof(float) * n_types * h->g.cells);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->nt[0], 0, bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->nt[1], 0, bytes, h->stream);
  if (e == cudaSuccess && h->d_smc && h->smc_planes < n_types) {
    // smart Monte Carlo: one table plane per type (rebuilt with the fields)
    float4* tab = nullptr;
    e = cudaMalloc((void**)&tab, sizeof(float4) * n_types * h->g.cells);
    if (e == cudaSuccess) {
      cudaFree(h->d_smc);
      h->d_smc = tab;
      h->smc_planes = n_types;
    }
  }
  if (e != cudaSuccess) {
    cudaFree(h->nt[0]);
    cudaFree(h->nt[1]);
    cudaFree(h->wt);
    h->nt[0] = h->nt[1] = nullptr;
    h->wt = nullptr;
    return cuda_fail(e, "type planes");
  }
  for (int k = 0; k < TYPES_MAX * TYPES_MAX; ++k) h->chiN_types[k] = 0.0;
  for (uint32_t i = 0; i < n_types; ++i)
    for (uint32_t j = 0; j < n_types; ++j) h->chiN_types[i * TYPES_MAX + j] = chiN[i * n_types + j];
  h->n_types = n_types;
  if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
  if (h->has_topo) set_topo_grid(h);
  if (h->has_topo) {   // the counts and fields of the current configuration
    soma_status st = update_fields(h);
    if (st != SOMA_OK) return st;
  }
  return sync(h);
}

soma_status soma_get_type_counts(soma_t* h, uint32_t* dst, size_t n, int dst_on_device) {
  if (!h || !dst) return fail(SOMA_EINVAL, "NULL argument");
  if (!h->n_types) return fail(SOMA_EINVAL, "no n_t types set: use soma_get_density");
  if (n != (size_t)h->n_types * h->g.cells)
    return fail(SOMA_EINVAL, "n=%zu, expected n_types*cells=%zu", n, (size_t)h->n_types * h->g.cells);
  SOMA_CUDA(cudaMemcpyAsync(dst, h->nt[h->host_sweep & 1], sizeof(uint32_t) * n,
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            h->stream));
  return sync(h);
}

soma_status soma_get_type_fields(soma_t* h, float* dst, size_t n, int dst_on_device) {
  if (!h || !dst) return fail(SOMA_EINVAL, "NULL argument");
  if (!h->n_types) return fail(SOMA_EINVAL, "no n_t types set: use soma_get_fields");
  if (n != (size_t)h->n_types * h->g.cells)
    return fail(SOMA_EINVAL, "n=%zu, expected n_types*cells=%zu", n, (size_t)h->n_types * h->g.cells);
  SOMA_CUDA(cudaMemcpyAsync(dst, h->wt, sizeof(float) * n,
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            h->stream));
  return sync(h);
}

soma_status soma_sort_molecules(soma_t* h, uint64_t* perm) {
  if (!h) return fail(SOMA_EINVAL, "handle is NULL");
  if (h->batched) return fail(SOMA_ESTATE, "a batch member keeps its labels");
  if (h->g.n_chains >= (1ull << 32)) return fail(SOMA_EINVAL, "labels need n_chains < 2^32");
  uint64_t n_pad = 1;
  while (n_pad < h->g.n_chains) n_pad <<= 1;
  float* stage = nullptr;
  uint64_t* keys = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&stage, sizeof(float) * 3 * h->plane, h->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&keys, sizeof(uint64_t) * n_pad, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(stage, h->pos, sizeof(float) * 3 * h->plane, cudaMemcpyDeviceToDevice,
                        h->stream);
  if (e == cudaSuccess)
    e = launch_sort_chains(h->g, stage, h->plane, h->pos, h->plane, keys, n_pad, h->sm_count,
                           h->stream);
  std::vector<uint64_t> k;
  if (e == cudaSuccess && (perm || h->d_arch)) {
    k.resize((size_t)h->g.n_chains);
    e = cudaMemcpyAsync(k.data(), keys, sizeof(uint64_t) * k.size(), cudaMemcpyDeviceToHost,
                        h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (stage) cudaFreeAsync(stage, h->stream);
  if (keys) cudaFreeAsync(keys, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "molecule sort");
  h->launches += 3;
  if (h->d_arch) {   // the architectures follow their molecules
    std::vector<uint8_t> a((size_t)h->g.n_chains), b(a.size());
    SOMA_CUDA(cudaMemcpyAsync(a.data(), h->d_arch, a.size(), cudaMemcpyDeviceToHost, h->stream));
    SOMA_CUDA(cudaStreamSynchronize(h->stream));
    for (size_t j = 0; j < b.size(); ++j) b[j] = a[k[j] & 0xFFFFFFFFull];
    SOMA_CUDA(cudaMemcpyAsync(h->d_arch, b.data(), b.size(), cudaMemcpyHostToDevice, h->stream));
    SOMA_CUDA(cudaStreamSynchronize(h->stream));
  }
  if (perm)
    for (size_t j = 0; j < k.size(); ++j) perm[j] = k[j] & 0xFFFFFFFFull;
  return sync(h);
}

soma_status soma_topology_sets(const uint32_t* words, uint64_t n_words, const uint32_t* start,
                               uint32_t n_arch, uint32_t N, uint8_t* sets, uint8_t* n_sets) {
  if (!words || !start || !sets || !n_sets) return fail(SOMA_EINVAL, "NULL argument");
  if (n_arch < 1 || n_arch > 256 || n_words < 2 || n_words > (1ull << 24) || N < 1)
    return fail(SOMA_EINVAL, "need 1..256 architectures in 2..2^24 words and N >= 1");
  TopologyTables T;
  const std::string why = topology_tables(words, n_words, start, n_arch, N, &T, TYPES_MAX);
  if (!why.empty()) return fail(SOMA_EINVAL, "%s", why.c_str());
  for (uint32_t a = 0; a < n_arch; ++a) {
    n_sets[a] = T.nsets[a];
    for (uint32_t i = 0; i < N; ++i)   // 0xFF: an absent slot (past the architecture's particles)
      sets[(size_t)a * N + i] =
          i < T.len[a] ? (uint8_t)((T.ptab[(size_t)a * 64 + i] >> 25) & 7u) : (uint8_t)0xFF;
  }
  return SOMA_OK;
}

soma_status soma_get_parameters(soma_t* h, soma_params* out) {
  if (!h || !out) return fail(SOMA_EINVAL, "NULL argument");
  const double N = (double)h->g.N;
  out->Re = h->Re;
  out->a = h->a64;
  out->K_b = h->K_b;
  out->b0 = h->g.N > 1 ? h->Re / std::sqrt(N - 1.0) : 0.0;
  out->rho_cell = h->rho_cell;
  // rho_0 R_e0^3 = (M / cells) * Re^3 in dL units
  out->sqrt_Nbar = h->rho_cell * h->Re * h->Re * h->Re / N;
  out->epsilon = out->b0 * out->b0 * out->b0 / std::sqrt(N * out->sqrt_Nbar * out->sqrt_Nbar);
  out->M = h->M;
  out->cells = h->g.cells;
  out->N_A = h->g.N_A;
  return SOMA_OK;
}

soma_status soma_check_bounded_wait(uint32_t limit, void* stream) {
  if (limit < 1) return fail(SOMA_EINVAL, "limit must be >= 1");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned* d = nullptr;
  SOMA_CUDA(cudaMalloc((void**)&d, sizeof(unsigned)));
  unsigned e = 0;
  cudaError_t c = cudaMemsetAsync(d, 0, sizeof(unsigned), st);
  if (c == cudaSuccess) c = launch_wait_probe(limit, d, st);
  if (c == cudaSuccess) c = cudaMemcpyAsync(&e, d, sizeof e, cudaMemcpyDeviceToHost, st);
  if (c == cudaSuccess) c = cudaStreamSynchronize(st);
  cudaFree(d);
  if (c != cudaSuccess) return cuda_fail(c, "bounded-wait probe");
  if (e & ERR_TIMEOUT) return fail(SOMA_ETIMEOUT, "the probe's wait gave up after %u polls (expected)", limit);
  return SOMA_OK;
}

soma_status soma_observables(soma_t* h, soma_obs* out) {
  if (!h || !out) return fail(SOMA_EINVAL, "NULL argument");
  const uint32_t* nn = h->n[h->host_sweep & 1];
  SOMA_CUDA(launch_observables(h->g, h->x(), h->y(), h->z(), nn, 1.0 / h->rho_cell,
                               h->desc.kappaN, h->desc.chiN, (int)h->desc.hamiltonian,
                               h->has_ext ? h->d_ext : nullptr, h->d_scratch, h->d_out, h->stream));
  h->launches += 3;
  if (h->has_topo) {   // the bonds of the architectures replace those of the linear chain
    SOMA_CUDA(launch_topology_bonds(h->g, h->x(), h->y(), h->z(), h->d_topo_pmask, h->d_arch,
                                    h->d_topo_len, h->d_scratch, h->d_out, h->stream));
    h->launches += 2;
  }
  if (h->n_types) {    // the non-bonded energy and largest count of the type planes
    SOMA_CUDA(launch_observables_types(types_args(h, 0), h->desc.kappaN, h->nt[h->host_sweep & 1],
                                       h->d_scratch, h->d_out, h->stream));
    h->launches += 2;
  }
  double r[5];
  unsigned long long c[2];
  SOMA_CUDA(cudaMemcpyAsync(r, h->d_out, sizeof r, cudaMemcpyDeviceToHost, h->stream));
  SOMA_CUDA(cudaMemcpyAsync(c, h->d_counters, sizeof c, cudaMemcpyDeviceToHost, h->stream));
  soma_status st = sync(h);
  if (st != SOMA_OK) return st;
  const double nch = (double)h->g.n_chains;
  const double nb = h->has_topo ? h->topo_bonds : nch * (double)(h->g.N > 1 ? h->g.N - 1 : 0);
  out->E_b = h->K_b * r[0];
  out->E_nb = h->rho_cell / (double)h->g.N * r[2];
  out->E_ext = r[4];
  out->E_tot = out->E_b + out->E_nb + out->E_ext;
  out->Re2 = r[1] / nch;
  out->Re2_rel = out->Re2 / (h->Re * h->Re);
  out->b2 = nb > 0 ? r[0] / nb : 0.0;
  out->accepted = c[1];
  out->sweeps = c[0];
  out->attempted = c[0] * h->M_real;
  out->max_cell = (uint32_t)r[3];
  out->reserved = 0;
  return SOMA_OK;
}

namespace {
// S(q) of the composition held in a packed grid (first type in bits 0-15,
// second in 16-31).
soma_status structure_factor_of(soma_t* h, const uint32_t* nn, const int32_t* m, size_t k,
                                double* out);
}  // namespace

soma_status soma_structure_factor(soma_t* h, const int32_t* m, size_t k, double* out) {
  if (!h || !m || !out) return fail(SOMA_EINVAL, "NULL argument");
  if (h->n_types) return fail(SOMA_EINVAL, "n_t types: use soma_structure_factor_types");
  if (k > 4096) return fail(SOMA_EINVAL, "k=%zu > 4096", k);
  if (k == 0) return SOMA_OK;
  return structure_factor_of(h, h->n[h->host_sweep & 1], m, k, out);
}

soma_status soma_structure_factor_types(soma_t* h, uint32_t ti, uint32_t tj, const int32_t* m,
                                        size_t k, double* out) {
  if (!h || !m || !out) return fail(SOMA_EINVAL, "NULL argument");
  const uint32_t T = h->n_types ? h->n_types : 2u;
  if (ti >= T || tj >= T || ti == tj)
    return fail(SOMA_EINVAL, "types %u, %u: need two different types below %u", ti, tj, T);
  if (k > 4096) return fail(SOMA_EINVAL, "k=%zu > 4096", k);
  if (k == 0) return SOMA_OK;
  // two types: the packed A | B grid (S of B - A equals S of A - B)
  if (!h->n_types) return structure_factor_of(h, h->n[h->host_sweep & 1], m, k, out);
  uint32_t* packed = nullptr;
  SOMA_CUDA(cudaMallocAsync((void**)&packed, sizeof(uint32_t) * h->g.cells, h->stream));
  cudaError_t e = launch_pack_type_pair(h->nt[h->host_sweep & 1], h->g.cells, ti, tj, packed,
                                        h->d_err, h->sm_count, h->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(packed, h->stream);
    return cuda_fail(e, "pack type pair");
  }
  soma_status st = structure_factor_of(h, packed, m, k, out);
  cudaFreeAsync(packed, h->stream);
  if (st != SOMA_OK) return st;
  return sync(h);
}

namespace {
soma_status structure_factor_of(soma_t* h, const uint32_t* nn, const int32_t* m, size_t k,
                                double* out) {
  const int nx = h->g.nx, ny = h->g.ny, nz = h->g.nz;
  const size_t T = (size_t)nx + ny + nz;
  const size_t need = (size_t)SQ_MAX * T * 2;
  if (h->tw_doubles < need) {
    cudaFree(h->d_tw);
    h->d_tw = nullptr;
    SOMA_CUDA(cudaMalloc((void**)&h->d_tw, sizeof(double) * need));
    h->tw_doubles = need;
  }
  std::vector<double> tw(need);
  const double two_pi = 6.283185307179586;
  for (size_t q0 = 0; q0 < k; q0 += SQ_MAX) {
    const int kk = (int)((k - q0) < (size_t)SQ_MAX ? (k - q0) : (size_t)SQ_MAX);
    for (int q = 0; q < kk; ++q) {
      const int n3[3] = {nx, ny, nz};
      size_t off = (size_t)q * T * 2;
      for (int d = 0; d < 3; ++d) {
        const long long md = m[3 * (q0 + q) + d];
        for (int c = 0; c < n3[d]; ++c) {
          long long r = (md * c) % n3[d];
          if (r < 0) r += n3[d];
          const double ph = two_pi * (double)r / (double)n3[d];
          tw[off++] = std::cos(ph);
          tw[off++] = -std::sin(ph);
        }
      }
    }
    SOMA_CUDA(cudaMemcpyAsync(h->d_tw, tw.data(), sizeof(double) * kk * T * 2,
                              cudaMemcpyHostToDevice, h->stream));
    SOMA_CUDA(launch_structure_factor(h->g, nn, h->d_tw, kk, h->d_scratch, h->d_out, h->stream));
    h->launches += 2;
    SOMA_CUDA(cudaMemcpyAsync(out + q0, h->d_out, sizeof(double) * kk, cudaMemcpyDeviceToHost,
                              h->stream));
    soma_status st = sync(h);
    if (st != SOMA_OK) return st;
  }
  return SOMA_OK;
}
}  // namespace

soma_status soma_get_sweep(soma_t* h, uint64_t* out) {
  if (!h || !out) return fail(SOMA_EINVAL, "NULL argument");
  *out = h->host_sweep;
  return SOMA_OK;
}

soma_status soma_set_sweep(soma_t* h, uint64_t sweep) {
  if (!h) return fail(SOMA_EINVAL, "handle is NULL");
  unsigned long long v = sweep;
  SOMA_CUDA(cudaMemcpyAsync(h->d_counters, &v, sizeof v, cudaMemcpyHostToDevice, h->stream));
  SOMA_CUDA(cudaStreamSynchronize(h->stream));
  h->host_sweep = sweep;
  h->shard_phase = 0;
  // the occupation buffer in use depends on the counter's parity
  if (h->n_types)
    SOMA_CUDA(cudaMemsetAsync(h->nt[(sweep + 1) & 1], 0,
                              sizeof(uint32_t) * h->n_types * h->g.cells, h->stream));
  else
    SOMA_CUDA(cudaMemsetAsync(h->n[(sweep + 1) & 1], 0, sizeof(uint32_t) * h->g.cells, h->stream));
  return update_fields(h);
}

soma_status soma_set_timing(soma_t* h, int on) {
  if (!h) return fail(SOMA_EINVAL, "handle is NULL");
  SOMA_CUDA(cudaStreamSynchronize(h->stream));
  for (auto& p : h->ev_pending) { h->ev_free.push_back(p.a); h->ev_free.push_back(p.b); }
  h->ev_pending.clear();
  h->timing = on != 0;
  if (h->timing) {
    h->t.ms_sweep = h->t.ms_fields = 0.0;
    h->t.sweep_launches = h->t.field_launches = 0;
  }
  return SOMA_OK;
}

soma_status soma_get_timing(soma_t* h, soma_timing* out) {
  if (!h || !out) return fail(SOMA_EINVAL, "NULL argument");
  SOMA_CUDA(cudaStreamSynchronize(h->stream));
  for (auto& p : h->ev_pending) {
    float ms = 0.f;
    SOMA_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
    if (p.kind == 0) h->t.ms_sweep += ms; else h->t.ms_fields += ms;
    h->ev_free.push_back(p.a);
    h->ev_free.push_back(p.b);
  }
  h->ev_pending.clear();
  *out = h->t;
  out->kernel_launches = h->launches;
  return SOMA_OK;
}

soma_status soma_proposal_set_weights(soma_t* h, const float* w, size_t n, int src_on_device) {
  if (!h || !w) return fail(SOMA_EINVAL, "NULL argument");
  if (n != SOMA_MLP_PARAMS) return fail(SOMA_EINVAL, "n=%zu, the network has %d parameters", n, SOMA_MLP_PARAMS);
  SOMA_CUDA(cudaMemcpyAsync(h->mlp_w, w, sizeof(float) * n,
                            src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            h->stream));
  SOMA_CUDA(launch_quantize(h->mlp_w, h->mlp_q, h->stream));
  SOMA_CUDA(cudaMemsetAsync(h->mlp_m, 0, sizeof(float) * n, h->stream));
  SOMA_CUDA(cudaMemsetAsync(h->mlp_v, 0, sizeof(float) * n, h->stream));
  h->train_step = 0;
  ++h->launches;
  if (!src_on_device) SOMA_CUDA(cudaStreamSynchronize(h->stream));
  return SOMA_OK;
}

soma_status soma_proposal_get_weights(soma_t* h, float* w, size_t n, int dst_on_device) {
  if (!h || !w) return fail(SOMA_EINVAL, "NULL argument");
  if (n != SOMA_MLP_PARAMS) return fail(SOMA_EINVAL, "n=%zu, the network has %d parameters", n, SOMA_MLP_PARAMS);
  SOMA_CUDA(cudaMemcpyAsync(w, h->mlp_w, sizeof(float) * n,
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            h->stream));
  return sync(h);
}

namespace {
TrainArgs train_args(soma_t* h) {
  TrainArgs t{};
  t.g = h->g;
  t.x = h->x();
  t.y = h->y();
  t.z = h->z();
  t.wA = h->w[0];
  t.wB = h->w[1];
  t.w = h->mlp_w;
  t.grad = h->mlp_g;
  t.sigma0 = (float)(h->a64 / std::sqrt(3.0));
  t.K_b = (float)h->K_b;
  return t;
}
}  // namespace

soma_status soma_proposal_grad(soma_t* h, const float* w, const uint32_t* samples, const float* xi,
                               uint32_t n, float* grad, float* J, float* log_alpha) {
  if (!h || !samples || !xi || !grad) return fail(SOMA_EINVAL, "NULL argument");
  TrainArgs t = train_args(h);
  if (w) t.w = w;
  t.grad = grad;
  t.J = J;
  t.log_alpha = log_alpha;
  t.samples = samples;
  t.xi = xi;
  t.n = n;
  SOMA_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * SOMA_MLP_PARAMS, h->stream));
  SOMA_CUDA(launch_esjd_grad(t, h->grid_dtype, h->sm_count, h->stream));
  h->launches += 1;
  return SOMA_OK;
}

soma_status soma_proposal_train(soma_t* h, const soma_train_cfg* cfg, soma_train_log* log) {
  if (h && h->pos_invalid) return fail(SOMA_ESTATE, "positions out of range: set valid positions first");
  if (!h || !cfg) return fail(SOMA_EINVAL, "NULL argument");
  if (cfg->batch < 1 || cfg->steps < 1) return fail(SOMA_EINVAL, "steps and batch must be >= 1");
  float* dJ = nullptr;
  float* dla = nullptr;
  SOMA_CUDA(cudaMallocAsync((void**)&dJ, sizeof(float) * cfg->batch, h->stream));
  SOMA_CUDA(cudaMallocAsync((void**)&dla, sizeof(float) * cfg->batch, h->stream));
  std::vector<float> hJ(cfg->batch), hla(cfg->batch);
  double first = 0.0, last = 0.0, acc_last = 0.0;
  const SweepArgs sa = sweep_args(h);
  const FieldArgs fa = field_args(h, 1);
  for (uint32_t k = 0; k < cfg->steps; ++k) {
    // trajectories of the plain method
    for (uint32_t c = 0; c < cfg->sweeps_between; ++c) {
      SOMA_CUDA(launch_sweep_uniform(sa, h->plain_shape, h->grid_dtype, h->stream));
      SOMA_CUDA(launch_fields(fa, h->d_err + 1, h->grid_dtype, h->sm_count, h->stream));
      ++h->host_sweep;
      h->launches += 2;
    }
    TrainArgs t = train_args(h);
    t.J = dJ;
    t.log_alpha = dla;
    t.n = cfg->batch;
    t.step = h->train_step;
    SOMA_CUDA(cudaMemsetAsync(h->mlp_g, 0, sizeof(float) * SOMA_MLP_PARAMS, h->stream));
    SOMA_CUDA(launch_esjd_grad(t, h->grid_dtype, h->sm_count, h->stream));
    ++h->train_step;
    SOMA_CUDA(launch_adam(h->mlp_w, h->mlp_m, h->mlp_v, h->mlp_g, h->mlp_q, cfg->lr, cfg->beta1,
                          cfg->beta2, cfg->eps, (int)h->train_step, 1.f / (float)cfg->batch,
                          h->stream));
    h->launches += 2;
    if (k == 0 || k + 1 == cfg->steps) {
      SOMA_CUDA(cudaMemcpyAsync(hJ.data(), dJ, sizeof(float) * cfg->batch, cudaMemcpyDeviceToHost, h->stream));
      SOMA_CUDA(cudaMemcpyAsync(hla.data(), dla, sizeof(float) * cfg->batch, cudaMemcpyDeviceToHost, h->stream));
      SOMA_CUDA(cudaStreamSynchronize(h->stream));
      double sj = 0.0, sa_ = 0.0;
      for (uint32_t b = 0; b < cfg->batch; ++b) {
        sj += hJ[b];
        sa_ += hla[b] >= 0.f ? 1.0 : std::exp((double)hla[b]);
      }
      if (k == 0) first = sj / cfg->batch;
      last = sj / cfg->batch;
      acc_last = sa_ / cfg->batch;
    }
  }
  cudaFreeAsync(dJ, h->stream);
  cudaFreeAsync(dla, h->stream);
  soma_status st = sync(h);
  if (st != SOMA_OK) return st;
  if (log) {
    log->mean_J_first = first;
    log->mean_J_last = last;
    log->mean_alpha_last = acc_last;
    log->steps_done = cfg->steps;
    log->reserved = 0;
  }
  return SOMA_OK;
}

soma_status soma_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n,
                        void* stream) {
  if (n && (!ctr || !key || !out)) return fail(SOMA_EINVAL, "NULL argument");
  SOMA_CUDA(launch_philox(ctr, key, out, n, (cudaStream_t)stream));
  return SOMA_OK;
}

soma_status soma_smc_draws(const uint32_t* words, float* out, size_t n, void* stream) {
  if (n && (!words || !out)) return fail(SOMA_EINVAL, "NULL argument");
  int dev = 0, sms = 1;
  SOMA_CUDA(cudaGetDevice(&dev));
  SOMA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SOMA_CUDA(launch_smc_draws(words, out, n, sms, (cudaStream_t)stream));
  return SOMA_OK;
}


// ---------------------------------------------------------------------------
// Batches of independent systems (one sweep launch + one field launch per cycle)
// ---------------------------------------------------------------------------
}  // extern "C"

struct soma_batch_t {
  std::vector<soma_t*> sys;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sm_count = 0;
  int grid_dtype = 0;
  BatchSys* d_sys = nullptr;
  BatchItem* d_items = nullptr;
  uint32_t n_items = 0, items_cap = 0;
  unsigned* d_aux = nullptr;  // [0] arrival counter, [1] error bits
  uint32_t total_cells = 0;
  BatchArgs args{};
  int block = 256, blocks_per_sm = 2, item_tiles = 0;
  cudaGraphExec_t graph = nullptr;
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_sweep, ev_field;
  soma_timing t{};
};

namespace {

void batch_release(soma_batch_t* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto& e : b->ev_sweep) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
  for (auto& e : b->ev_field) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
  for (soma_t* h : b->sys) {
    h->batched = false;
    h->own_stream = false;
    release(h);
  }
  cudaFree(b->d_sys);
  cudaFree(b->d_items);
  cudaFree(b->d_aux);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// The work items of a batch whose member k has nt[k] tiles, for a sweep
// launch of grid blocks (block j takes items j, j + grid, j + 2 grid, ...).
// item_tiles > 0: runs of item_tiles tiles of each member in turn.
// item_tiles == 0: one contiguous range of the members' concatenated tiles per
// block, equal to within a tile, cut at member boundaries into pieces; piece
// r of block j sits at item r * grid + j, and blocks with fewer pieces get
// empty items.
std::vector<BatchItem> batch_plan(const std::vector<uint32_t>& nt, uint32_t grid, int item_tiles) {
  std::vector<BatchItem> items;
  if (item_tiles > 0) {
    for (uint32_t k = 0; k < nt.size(); ++k)
      for (uint32_t t0 = 0; t0 < nt[k]; t0 += (uint32_t)item_tiles)
        items.push_back({k, t0, std::min(nt[k], t0 + (uint32_t)item_tiles)});
    return items;
  }
  std::vector<uint64_t> begin(nt.size() + 1, 0);
  for (uint32_t k = 0; k < nt.size(); ++k) begin[k + 1] = begin[k] + nt[k];
  const uint64_t total = begin.back();
  std::vector<std::vector<BatchItem>> per(grid);
  size_t rounds = 1;
  uint32_t k = 0;
  for (uint32_t j = 0; j < grid; ++j) {
    uint64_t g0 = total * j / grid;
    const uint64_t g1 = total * (j + 1) / grid;
    while (g0 < g1) {
      while (begin[k + 1] <= g0) ++k;
      const uint64_t e = std::min(g1, begin[k + 1]);
      per[j].push_back({k, (uint32_t)(g0 - begin[k]), (uint32_t)(e - begin[k])});
      g0 = e;
    }
    rounds = std::max(rounds, per[j].size());
  }
  items.assign(rounds * grid, BatchItem{0u, 0u, 0u});
  for (uint32_t j = 0; j < grid; ++j)
    for (size_t r = 0; r < per[j].size(); ++r) items[r * grid + j] = per[j][r];
  return items;
}

soma_status batch_items(soma_batch_t* b, int item_tiles) {
  std::vector<uint32_t> nt(b->sys.size());
  for (size_t k = 0; k < b->sys.size(); ++k) nt[k] = (uint32_t)b->sys[k]->shape.n_tiles;
  const std::vector<BatchItem> items =
      batch_plan(nt, (uint32_t)(b->sm_count * b->blocks_per_sm), item_tiles);
  if (items.size() > b->items_cap) {
    cudaFree(b->d_items);
    b->d_items = nullptr;
    SOMA_CUDA(cudaMalloc((void**)&b->d_items, sizeof(BatchItem) * items.size()));
    b->items_cap = (uint32_t)items.size();
  }
  SOMA_CUDA(cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * items.size(),
                            cudaMemcpyHostToDevice, b->stream));
  SOMA_CUDA(cudaStreamSynchronize(b->stream));
  b->n_items = (uint32_t)items.size();
  b->item_tiles = item_tiles;
  b->args.items = b->d_items;
  b->args.n_items = b->n_items;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  return SOMA_OK;
}

soma_status batch_cycle(soma_batch_t* b) {
  cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
  if (b->timing)
    for (auto& x : e) SOMA_CUDA(cudaEventCreate(&x));
  if (b->timing) SOMA_CUDA(cudaEventRecord(e[0], b->stream));
  SOMA_CUDA(launch_sweep_batch(b->args, b->sm_count * b->blocks_per_sm, b->block, b->grid_dtype,
                               b->stream));
  if (b->timing) {
    SOMA_CUDA(cudaEventRecord(e[1], b->stream));
    SOMA_CUDA(cudaEventRecord(e[2], b->stream));
  }
  SOMA_CUDA(launch_fields_batch(b->args, b->total_cells, b->d_aux, b->d_aux + 1, b->grid_dtype,
                                b->sm_count, b->stream));
  if (b->timing) {
    SOMA_CUDA(cudaEventRecord(e[3], b->stream));
    b->ev_sweep.push_back({e[0], e[1]});
    b->ev_field.push_back({e[2], e[3]});
  }
  b->t.sweep_launches++;
  b->t.field_launches++;
  b->t.kernel_launches += 2;
  for (soma_t* h : b->sys) ++h->host_sweep;
  return SOMA_OK;
}

soma_status batch_graph(soma_batch_t* b) {
  cudaGraph_t gr = nullptr;
  SOMA_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (uint32_t k = 0; k < GRAPH_CHUNK && e == cudaSuccess; ++k) {
    e = launch_sweep_batch(b->args, b->sm_count * b->blocks_per_sm, b->block, b->grid_dtype,
                           b->stream);
    if (e == cudaSuccess)
      e = launch_fields_batch(b->args, b->total_cells, b->d_aux, b->d_aux + 1, b->grid_dtype,
                              b->sm_count, b->stream);
  }
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &gr);
  if (e != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return cuda_fail(e, "batch graph capture"); }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&b->graph, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) { b->graph = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
  return SOMA_OK;
}

soma_status batch_collect_timing(soma_batch_t* b) {
  SOMA_CUDA(cudaStreamSynchronize(b->stream));
  for (auto& e : b->ev_sweep) {
    float ms = 0.f;
    SOMA_CUDA(cudaEventElapsedTime(&ms, e.first, e.second));
    b->t.ms_sweep += ms;
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto& e : b->ev_field) {
    float ms = 0.f;
    SOMA_CUDA(cudaEventElapsedTime(&ms, e.first, e.second));
    b->t.ms_fields += ms;
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  b->ev_sweep.clear();
  b->ev_field.clear();
  return SOMA_OK;
}

}  // namespace

extern "C" {

soma_status soma_batch_create(const soma_system_desc* descs, uint32_t n, void* stream,
                              soma_batch_t** out) {
  if (!out || !descs) return fail(SOMA_EINVAL, "NULL argument");
  *out = nullptr;
  if (n < 1 || n > SOMA_BATCH_MAX) return fail(SOMA_EINVAL, "batch size %u outside 1..%d", n, SOMA_BATCH_MAX);
  for (uint32_t k = 0; k < n; ++k) {
    soma_status st = validate(descs + k);
    if (st != SOMA_OK) return st;
    const soma_system_desc& d = descs[k];
    if (d.N % 2 != 0 || d.N > 64)
      return fail(SOMA_EINVAL, "batch member %u: N=%u (a batch takes even N <= 64)", k, d.N);
    if (d.move != SOMA_MOVE_UNIFORM)
      return fail(SOMA_EINVAL, "batch member %u: only uniform moves are batched", k);
    if (d.set_order == SOMA_ITERATION_MOLECULE)
      return fail(SOMA_EINVAL, "batch member %u: a batch runs the SET scheme", k);
    if (d.seed != descs[0].seed)
      return fail(SOMA_EINVAL, "batch member %u: all members share one seed (use replica_id)", k);
    if (d.grid_dtype != descs[0].grid_dtype)
      return fail(SOMA_EINVAL, "batch member %u: all members share one grid_dtype", k);
    if (d.n_chains * d.N >= (1ull << 32)) return fail(SOMA_EINVAL, "batch member %u: M >= 2^32", k);
    if (d.n_chains_total) return fail(SOMA_EINVAL, "batch member %u: a batch holds whole systems", k);
  }
  soma_batch_t* b = new (std::nothrow) soma_batch_t();
  if (!b) return fail(SOMA_ENOMEM, "host allocation failed");
  cudaError_t e = cudaSuccess;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaStreamCreate"); }
    b->own_stream = true;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
  b->grid_dtype = descs[0].grid_dtype;
  std::vector<BatchSys> table(n);
  uint32_t cells = 0;
  for (uint32_t k = 0; k < n; ++k) {
    soma_system_desc d = descs[k];
    d.stream = b->stream;
    soma_t* h = nullptr;
    soma_status st = soma_create(&d, &h);
    if (st != SOMA_OK) {
      char m[ERR_LEN];
      memcpy(m, g_last_error, ERR_LEN);
      batch_release(b);
      return fail(st, "batch member %u: %s", k, m);
    }
    h->batched = true;
    b->sys.push_back(h);
    BatchSys& S = table[k];
    S.g = h->g;
    S.x = h->x();
    S.y = h->y();
    S.z = h->z();
    S.wA = h->w[0];
    S.wB = h->w[1];
    S.n0 = h->n[0];
    S.n1 = h->n[1];
    S.counters = h->d_counters;
    S.a = h->a32;
    S.K_b = (float)h->K_b;
    S.G = h->shape.G;
    S.full_tiles = (uint32_t)(h->g.n_chains / h->shape.G);
    S.last_rows = (uint32_t)(h->g.n_chains % h->shape.G) * h->g.N;
    S.cell_begin = cells;
    S.inv_rho = (float)(1.0 / h->rho_cell);
    S.kappa0 = (float)(h->desc.kappaN / (double)h->desc.N);
    S.half_chi0 = (float)(0.5 * h->desc.chiN / (double)h->desc.N);
    S.set_order_random = h->desc.set_order == SOMA_SET_ORDER_RANDOM;
    S.hamiltonian = (int)h->desc.hamiltonian;
    cells += h->g.cells;
    if (cells < h->g.cells) { batch_release(b); return fail(SOMA_EINVAL, "batch grids exceed 2^32 cells"); }
  }
  b->total_cells = cells;
#define BCK(call) do { e = (call); if (e != cudaSuccess) { batch_release(b); return cuda_fail(e, #call); } } while (0)
  BCK(cudaMalloc((void**)&b->d_sys, sizeof(BatchSys) * n));
  BCK(cudaMalloc((void**)&b->d_aux, sizeof(unsigned) * 2));
  BCK(cudaMemsetAsync(b->d_aux, 0, sizeof(unsigned) * 2, b->stream));
  BCK(cudaMemcpyAsync(b->d_sys, table.data(), sizeof(BatchSys) * n, cudaMemcpyHostToDevice, b->stream));
#undef BCK
  b->args.sys = b->d_sys;
  b->args.n_sys = n;
  b->args.keys = b->sys[0]->g;
  b->args.d_sweep = b->sys[0]->d_counters;
  const int fit = batch_kernel_blocks_per_sm(b->block, b->grid_dtype);
  b->blocks_per_sm = fit < 1 ? 1 : (fit < 3 ? fit : 3);
  soma_status st = batch_items(b, b->item_tiles);
  if (st != SOMA_OK) { KeepError keep; batch_release(b); return st; }
  *out = b;
  return SOMA_OK;
}

soma_status soma_batch_destroy(soma_batch_t* b) {
  if (!b) return SOMA_OK;
  batch_release(b);
  return SOMA_OK;
}

soma_status soma_batch_system(soma_batch_t* b, uint32_t i, soma_t** out) {
  if (!b || !out) return fail(SOMA_EINVAL, "NULL argument");
  if (i >= b->sys.size()) return fail(SOMA_EINVAL, "member %u of a batch of %zu", i, b->sys.size());
  *out = b->sys[i];
  return SOMA_OK;
}

soma_status soma_batch_sweep(soma_batch_t* b, uint32_t n) {
  if (!b) return fail(SOMA_EINVAL, "batch is NULL");
  for (soma_t* h : b->sys)
    if (h->pos_invalid) return fail(SOMA_ESTATE, "a member holds positions out of range");
  uint32_t done = 0;
  if (!b->timing && n >= GRAPH_CHUNK) {
    if (!b->graph) {
      soma_status st = batch_graph(b);
      if (st != SOMA_OK) return st;
    }
    while (n - done >= GRAPH_CHUNK) {
      SOMA_CUDA(cudaGraphLaunch(b->graph, b->stream));
      b->t.sweep_launches += GRAPH_CHUNK;
      b->t.field_launches += GRAPH_CHUNK;
      b->t.kernel_launches += 2 * GRAPH_CHUNK;
      for (soma_t* h : b->sys) h->host_sweep += GRAPH_CHUNK;
      done += GRAPH_CHUNK;
    }
  }
  for (; done < n; ++done) {
    soma_status st = batch_cycle(b);
    if (st != SOMA_OK) return st;
  }
  return SOMA_OK;
}

soma_status soma_batch_sync(soma_batch_t* b) {
  if (!b) return fail(SOMA_EINVAL, "batch is NULL");
  SOMA_CUDA(cudaStreamSynchronize(b->stream));
  unsigned err = 0;
  SOMA_CUDA(cudaMemcpy(&err, b->d_aux + 1, sizeof err, cudaMemcpyDeviceToHost));
  if (err & ERR_OVERFLOW) return fail(SOMA_EOVERFLOW, "a 16-bit occupation number reached 0xC000");
  return SOMA_OK;
}

soma_status soma_batch_set_timing(soma_batch_t* b, int on) {
  if (!b) return fail(SOMA_EINVAL, "batch is NULL");
  soma_status st = batch_collect_timing(b);
  if (st != SOMA_OK) return st;
  b->timing = on != 0;
  if (b->timing) {
    b->t.ms_sweep = b->t.ms_fields = 0.0;
    b->t.sweep_launches = b->t.field_launches = 0;
  }
  return SOMA_OK;
}

soma_status soma_batch_get_timing(soma_batch_t* b, soma_timing* out) {
  if (!b || !out) return fail(SOMA_EINVAL, "NULL argument");
  soma_status st = batch_collect_timing(b);
  if (st != SOMA_OK) return st;
  *out = b->t;
  return SOMA_OK;
}

soma_status soma_batch_autotune(soma_batch_t* b, uint32_t cycles_per_candidate,
                                soma_tune_entry* table, uint32_t table_len, uint32_t* n_written) {
  if (!b) return fail(SOMA_EINVAL, "batch is NULL");
  if (cycles_per_candidate < 1) cycles_per_candidate = 1;
  const int blocks[3] = {128, 256, 512};
  const int items[4] = {16, 64, 256, 0};
  std::vector<soma_tune_entry> res;
  cudaEvent_t e0, e1;
  SOMA_CUDA(cudaEventCreate(&e0));
  SOMA_CUDA(cudaEventCreate(&e1));
  const bool was_timing = b->timing;
  b->timing = false;
  soma_tune_entry best{};
  best.ms_per_cycle = 1e30;
  for (int it : items) {
    soma_status st = batch_items(b, it);
    if (st != SOMA_OK) return st;
    for (int blk : blocks) {
      const int fit = batch_kernel_blocks_per_sm(blk, b->grid_dtype);
      for (int bps = 1; bps <= fit && bps <= 8; ++bps) {
        b->block = blk;
        b->blocks_per_sm = bps;
        if (it == 0) {  // the balanced split depends on the grid
          st = batch_items(b, 0);
          if (st != SOMA_OK) return st;
        }
        st = batch_cycle(b);  // warm-up with this shape
        if (st != SOMA_OK) return st;
        SOMA_CUDA(cudaEventRecord(e0, b->stream));
        for (uint32_t c = 0; c < cycles_per_candidate; ++c) {
          st = batch_cycle(b);
          if (st != SOMA_OK) return st;
        }
        SOMA_CUDA(cudaEventRecord(e1, b->stream));
        SOMA_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        SOMA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        soma_tune_entry r{blk, bps, it, 0, (double)ms / cycles_per_candidate};
        res.push_back(r);
        if (r.ms_per_cycle < best.ms_per_cycle) best = r;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->timing = was_timing;
  b->block = best.block;
  b->blocks_per_sm = best.blocks_per_sm;
  soma_status st = batch_items(b, best.item_tiles);
  if (st != SOMA_OK) return st;
  if (table)
    for (uint32_t k = 0; k < table_len && k < res.size(); ++k) table[k] = res[k];
  if (n_written) *n_written = (uint32_t)res.size();
  return SOMA_OK;
}

soma_status soma_batch_plan(const uint32_t* member_tiles, uint32_t n_members, uint32_t grid,
                            int32_t item_tiles, uint32_t* items, size_t capacity, size_t* n_items) {
  if (!member_tiles || !n_items) return fail(SOMA_EINVAL, "NULL argument");
  if (n_members < 1 || n_members > SOMA_BATCH_MAX)
    return fail(SOMA_EINVAL, "n_members=%u outside 1..%d", n_members, SOMA_BATCH_MAX);
  if (item_tiles < 0) return fail(SOMA_EINVAL, "item_tiles=%d < 0", (int)item_tiles);
  if (item_tiles == 0 && (grid < 1 || grid > (1u << 20)))
    return fail(SOMA_EINVAL, "grid=%u outside 1..2^20", grid);
  std::vector<uint32_t> nt(member_tiles, member_tiles + n_members);
  const std::vector<BatchItem> plan = batch_plan(nt, grid, item_tiles);
  *n_items = plan.size();
  if (!items) return SOMA_OK;
  if (capacity < plan.size())
    return fail(SOMA_EINVAL, "capacity %zu < %zu items", capacity, plan.size());
  for (size_t i = 0; i < plan.size(); ++i) {
    items[3 * i] = plan[i].sys;
    items[3 * i + 1] = plan[i].t0;
    items[3 * i + 2] = plan[i].t1;
  }
  return SOMA_OK;
}

soma_status soma_batch_set_shape(soma_batch_t* b, const soma_tune_entry* shape) {
  if (!b || !shape) return fail(SOMA_EINVAL, "NULL argument");
  if (shape->block < 32 || shape->block > 1024 || shape->block % 32 != 0)
    return fail(SOMA_EINVAL, "block=%d: a multiple of 32 in 32..1024", (int)shape->block);
  const int fit = batch_kernel_blocks_per_sm(shape->block, b->grid_dtype);
  if (shape->blocks_per_sm < 1 || shape->blocks_per_sm > fit)
    return fail(SOMA_EINVAL, "blocks_per_sm=%d: 1..%d fit on an SM with block=%d",
                (int)shape->blocks_per_sm, fit, (int)shape->block);
  if (shape->item_tiles < 0) return fail(SOMA_EINVAL, "item_tiles=%d < 0", (int)shape->item_tiles);
  b->block = shape->block;
  b->blocks_per_sm = shape->blocks_per_sm;
  return batch_items(b, shape->item_tiles);
}

soma_status soma_batch_get_shape(soma_batch_t* b, soma_tune_entry* out) {
  if (!b || !out) return fail(SOMA_EINVAL, "NULL argument");
  *out = soma_tune_entry{b->block, b->blocks_per_sm, b->item_tiles, 0, 0.0};
  return SOMA_OK;
}

}  // extern "C"
