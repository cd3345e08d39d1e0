// capi.cu -- the library's C ABI (declared in include/fv.h): handle
// lifetime, host->device upload, the time loop as captured CUDA graphs, and
// status reporting.  Every entry point converts exceptions into a status code
// and a thread-local message.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fv.h"
#include "fv_internal.h"
#include "kernels.h"

namespace {

thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define FV_CUDA(expr)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw fv::Error{FV_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)};     \
  } while (0)

template <typename F>
int guarded(F&& f) {
  try {
    f();
    return FV_OK;
  } catch (const fv::Error& e) {
    return set_error(e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return set_error(FV_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return set_error(FV_EINVAL, e.what());
  }
}

[[noreturn]] void invalid(const std::string& msg) { throw fv::Error{FV_EINVAL, msg}; }

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

template <typename T>
void dev_free(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// Steps per captured graph: a multiple of 6 so that the ping-pong buffers
// (period 2) and the rotating dt slots (period 3) are back in their starting
// roles after each graph, and the same graph can be replayed.
constexpr int64_t kGraphSteps = 96;

}  // namespace

namespace fv {
// Sets this thread's fv_last_error message (for entry points in other files).
int record_error(int code, const std::string& msg) { return set_error(code, msg); }
}  // namespace fv

struct fv_closure;  // defined with the learned closure

struct fv_mesh {
  fv::HostMesh h;
  int32_t precision = FV_F32;
  double uinf_prim[4] = {1.0, 0.0, 0.0, 1.0};  // rho, u, v, p
  // device side
  int device = -1;
  bool dirty = true;
  int64_t dev_n = -1;
  int4* d_nbr = nullptr;
  void* d_geom = nullptr;
  double* d_vol = nullptr;
  void* d_work = nullptr;  // ping-pong partner of the caller's state / RK2 stage
  uint2* d_lo = nullptr;        // FP32 compensated update: remainder of the state
  uint2* d_lo_stage = nullptr;  // ... and of the RK2 stage state
  bool compensated = true;      // FP32 meshes only
  fv::LoopScalars* d_scal = nullptr;
  double* d_partials = nullptr;
  cudaStream_t cap_stream = nullptr;
  // cached graph of kGraphSteps steps
  cudaGraphExec_t graph = nullptr;
  const void* g_U = nullptr;
  int32_t g_scheme = -1;
  double g_cfl = 0.0, g_tstop = 0.0;
  const fv_closure* g_closure = nullptr;
  bool g_comp = false;
  int last_t_slot = 0;
  bool stepped = false;

  bool f64() const { return precision == FV_F64; }
  size_t rec_bytes() const { return f64() ? 32 : 16; }
  bool use_lo() const { return !f64() && compensated; }

  void uinf_conserved(double* U) const {
    const double r = uinf_prim[0], u = uinf_prim[1], v = uinf_prim[2], p = uinf_prim[3];
    U[0] = r;
    U[1] = r * u;
    U[2] = r * v;
    U[3] = p / (1.4 - 1.0) + 0.5 * r * (u * u + v * v);
  }

  void drop_graph() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    g_U = nullptr;
  }

  void free_device() {
    drop_graph();
    dev_free(d_nbr);
    dev_free(d_geom);
    dev_free(d_vol);
    dev_free(d_work);
    dev_free(d_lo);
    dev_free(d_lo_stage);
    dev_free(d_scal);
    dev_free(d_partials);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
    dev_n = -1;
    dirty = true;
  }
};

namespace {

void ensure_device(fv_mesh* m, cudaStream_t s) {
  int dev = 0;
  FV_CUDA(cudaGetDevice(&dev));
  if (m->device >= 0 && m->device != dev && m->dev_n >= 0)
    invalid("mesh was uploaded to device " + std::to_string(m->device) +
            " but the current device is " + std::to_string(dev));
  if (!m->dirty && m->dev_n == m->h.n) return;
  const int64_t n = m->h.n;
  if (m->dev_n != n) {
    m->free_device();
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    FV_CUDA(cudaMalloc((void**)&m->d_nbr, nn * sizeof(int4)));
    FV_CUDA(cudaMalloc(&m->d_geom, nn * 2 * m->rec_bytes()));
    FV_CUDA(cudaMalloc((void**)&m->d_vol, nn * sizeof(double)));
    FV_CUDA(cudaMalloc(&m->d_work, nn * m->rec_bytes()));
    if (!m->f64()) {
      FV_CUDA(cudaMalloc((void**)&m->d_lo, nn * sizeof(uint2)));
      FV_CUDA(cudaMalloc((void**)&m->d_lo_stage, nn * sizeof(uint2)));
    }
    FV_CUDA(cudaMalloc((void**)&m->d_scal, sizeof(fv::LoopScalars)));
    FV_CUDA(cudaMalloc((void**)&m->d_partials, fv::kTotalsBlocks * 4 * sizeof(double)));
    FV_CUDA(cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
    m->dev_n = n;
  }
  m->drop_graph();
  std::vector<int4> nbr(n);
  for (int64_t c = 0; c < n; ++c)
    nbr[c] = make_int4(m->h.nbr[3 * c], m->h.nbr[3 * c + 1], m->h.nbr[3 * c + 2], 0);
  std::vector<double> geom(8 * n);
  for (int64_t c = 0; c < n; ++c) {
    for (int k = 0; k < 6; ++k) geom[8 * c + k] = m->h.nrm[6 * c + k];
    geom[8 * c + 6] = 1.0 / m->h.vol[c];
    geom[8 * c + 7] = m->h.inradius[c];
  }
  if (n > 0) {
    FV_CUDA(cudaMemcpyAsync(m->d_nbr, nbr.data(), n * sizeof(int4), cudaMemcpyHostToDevice, s));
    FV_CUDA(cudaMemcpyAsync(m->d_vol, m->h.vol.data(), n * sizeof(double), cudaMemcpyHostToDevice,
                            s));
    if (m->f64()) {
      FV_CUDA(cudaMemcpyAsync(m->d_geom, geom.data(), 8 * n * sizeof(double),
                              cudaMemcpyHostToDevice, s));
    } else {
      std::vector<float> g32(geom.begin(), geom.end());
      FV_CUDA(cudaMemcpyAsync(m->d_geom, g32.data(), 8 * n * sizeof(float),
                              cudaMemcpyHostToDevice, s));
      FV_CUDA(cudaStreamSynchronize(s));  // g32 is a local staging buffer
    }
  }
  FV_CUDA(cudaStreamSynchronize(s));
  m->device = dev;
  m->dirty = false;
}

fv::StepArgs base_args(const fv_mesh* m) {
  fv::StepArgs a{};
  a.nbr = m->d_nbr;
  a.geom = m->d_geom;
  a.n = m->h.n;
  m->uinf_conserved(a.uinf);
  a.err = &m->d_scal->err;
  return a;
}

// Enqueues steps j0 .. j0+count-1 of a loop on stream s.
void enqueue_steps(fv_mesh* m, void* U, int64_t j0, int64_t count, double cfl, double t_stop,
                   int32_t scheme, cudaStream_t s) {
  fv::LoopScalars* sc = m->d_scal;
  for (int64_t j = j0; j < j0 + count; ++j) {
    fv::StepArgs a = base_args(m);
    a.bmin_read = &sc->bmin[j % 3];
    a.bmin_write = &sc->bmin[(j + 1) % 3];
    a.bmin_reset = &sc->bmin[(j + 2) % 3];
    a.t_read = &sc->t[j % 2];
    a.t_write = &sc->t[(j + 1) % 2];
    a.cfl = cfl;
    a.t_stop = t_stop;
    if (m->use_lo()) {
      a.lo = m->d_lo;
      a.lo_stage = m->d_lo_stage;
    }
    if (scheme == FV_SCHEME_FE) {
      const bool even = (j % 2) == 0;
      a.U = even ? U : m->d_work;
      a.out = even ? m->d_work : U;
      FV_CUDA(fv::launch_step(m->f64(), fv::kModeFE, a, s));
    } else {
      a.U = U;
      a.out = m->d_work;
      FV_CUDA(fv::launch_step(m->f64(), fv::kModeRK2a, a, s));
      a.U = m->d_work;
      a.Ubase = U;
      a.out = U;
      FV_CUDA(fv::launch_step(m->f64(), fv::kModeRK2b, a, s));
    }
  }
}

void capture_graph(fv_mesh* m, void* U, double cfl, double t_stop, int32_t scheme,
                   const fv_closure* cl) {
  m->drop_graph();
  cudaGraph_t g = nullptr;
  FV_CUDA(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
  try {
    enqueue_steps(m, U, 0, kGraphSteps, cfl, t_stop, scheme, m->cap_stream);
  } catch (...) {
    cudaStreamEndCapture(m->cap_stream, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  FV_CUDA(cudaStreamEndCapture(m->cap_stream, &g));
  cudaError_t e = cudaGraphInstantiate(&m->graph, g, 0);
  cudaGraphDestroy(g);
  FV_CUDA(e);
  m->g_U = U;
  m->g_scheme = scheme;
  m->g_cfl = cfl;
  m->g_tstop = t_stop;
  m->g_closure = cl;
  m->g_comp = m->use_lo();
}

void read_status(fv_mesh* m, cudaStream_t s, double* t_adv, bool check) {
  fv::LoopScalars h{};
  FV_CUDA(cudaMemcpyAsync(&h, m->d_scal, sizeof h, cudaMemcpyDeviceToHost, s));
  FV_CUDA(cudaStreamSynchronize(s));
  if (t_adv) *t_adv = h.t[m->last_t_slot];
  if (check && h.err) throw fv::Error{FV_ENONFINITE, "a step produced a non-finite state or "
                                                     "non-positive density or pressure"};
}

void check_mesh(const fv_mesh* m) {
  if (!m) invalid("null mesh");
}

}  // namespace

extern "C" {

const char* fv_last_error(void) { return g_last_error.c_str(); }

int32_t fv_abi_version(void) { return 1; }

int fv_mesh_create(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
                   const int32_t* node_canon, const int32_t* bnd_edges, int64_t n_bnd,
                   int32_t default_bc, int32_t precision, fv_mesh** out) {
  return guarded([&] {
    if (!out) invalid("null out");
    *out = nullptr;
    if (precision != FV_F32 && precision != FV_F64) invalid("precision must be FV_F32 or FV_F64");
    fv_mesh* m = new fv_mesh();
    try {
      fv::build_host_mesh(xy, n_nodes, tri, n_tri, node_canon, bnd_edges, n_bnd, default_bc, m->h);
    } catch (...) {
      delete m;
      throw;
    }
    m->precision = precision;
    *out = m;
  });
}

int fv_mesh_destroy(fv_mesh* mesh) {
  return guarded([&] {
    if (!mesh) return;
    if (mesh->dev_n >= 0) {
      int cur = 0;
      cudaGetDevice(&cur);
      cudaSetDevice(mesh->device);
      cudaDeviceSynchronize();
      mesh->free_device();
      cudaSetDevice(cur);
    }
    delete mesh;
  });
}

int fv_mesh_info(const fv_mesh* mesh, int64_t* n_cells, int32_t* precision) {
  return guarded([&] {
    check_mesh(mesh);
    if (n_cells) *n_cells = mesh->h.n;
    if (precision) *precision = mesh->precision;
  });
}

int fv_set_freestream(fv_mesh* mesh, double rho, double u, double v, double p) {
  return guarded([&] {
    check_mesh(mesh);
    if (!(rho > 0.0) || !(p > 0.0) || !std::isfinite(rho) || !std::isfinite(p) ||
        !std::isfinite(u) || !std::isfinite(v))
      invalid("free stream needs finite rho > 0, p > 0 and finite velocity");
    mesh->uinf_prim[0] = rho;
    mesh->uinf_prim[1] = u;
    mesh->uinf_prim[2] = v;
    mesh->uinf_prim[3] = p;
    mesh->drop_graph();  // the free stream is a kernel argument baked into the graph
  });
}

int fv_renumber(fv_mesh* mesh, int32_t order, uint64_t seed, int32_t* perm_out) {
  return guarded([&] {
    check_mesh(mesh);
    std::vector<int32_t> perm;
    switch (order) {
      case FV_ORDER_IDENTITY:
        perm.resize(mesh->h.n);
        for (int64_t i = 0; i < mesh->h.n; ++i) perm[i] = (int32_t)i;
        break;
      case FV_ORDER_SHUFFLE: perm = fv::order_shuffle(mesh->h.n, seed); break;
      case FV_ORDER_RCM: perm = fv::order_rcm(mesh->h); break;
      case FV_ORDER_HILBERT: perm = fv::order_hilbert(mesh->h); break;
      default: invalid("unknown order");
    }
    fv::apply_permutation(mesh->h, perm);
    if (perm_out) std::memcpy(perm_out, perm.data(), perm.size() * sizeof(int32_t));
    mesh->dirty = true;
    mesh->drop_graph();
  });
}

int fv_mesh_diagnostics(const fv_mesh* mesh, int64_t* bandwidth, int64_t* serial_bandwidth) {
  return guarded([&] {
    check_mesh(mesh);
    if (bandwidth) *bandwidth = fv::graph_bandwidth(mesh->h);
    if (serial_bandwidth) *serial_bandwidth = fv::serial_bandwidth(mesh->h);
  });
}

int fv_mesh_export(const fv_mesh* mesh, int32_t* nbr, double* normals, double* area) {
  return guarded([&] {
    check_mesh(mesh);
    const int64_t n = mesh->h.n;
    if (nbr) std::memcpy(nbr, mesh->h.nbr.data(), 3 * n * sizeof(int32_t));
    if (normals) std::memcpy(normals, mesh->h.nrm.data(), 6 * n * sizeof(double));
    if (area) std::memcpy(area, mesh->h.vol.data(), n * sizeof(double));
  });
}

int fv_mesh_set_compensation(fv_mesh* mesh, int32_t enable) {
  return guarded([&] {
    check_mesh(mesh);
    if (mesh->f64() && enable) invalid("compensated update applies to FV_F32 meshes only");
    mesh->compensated = enable != 0;
    mesh->drop_graph();
  });
}

int fv_mesh_upload(fv_mesh* mesh, void* stream) {
  return guarded([&] {
    check_mesh(mesh);
    ensure_device(mesh, as_stream(stream));
  });
}

int fv_step(fv_mesh* mesh, void* U, int64_t nsteps, double cfl, double t_stop, int32_t scheme,
            const fv_closure* closure, void* stream, double* t_advanced) {
  return guarded([&] {
    check_mesh(mesh);
    if (nsteps < 0) invalid("nsteps < 0");
    if (scheme != FV_SCHEME_FE && scheme != FV_SCHEME_RK2) invalid("unknown scheme");
    if (!std::isfinite(cfl) || cfl == 0.0) invalid("cfl must be finite and non-zero");
    if (!std::isfinite(t_stop)) invalid("t_stop must be finite");
    if (closure) invalid("learned closure is not available in this build");
    if (!U && nsteps > 0 && mesh->h.n > 0) invalid("null state");
    cudaStream_t s = as_stream(stream);
    ensure_device(mesh, s);
    const int64_t n = mesh->h.n;
    FV_CUDA(fv::launch_init_scalars(mesh->d_scal, s));
    mesh->last_t_slot = 0;
    mesh->stepped = true;
    if (n > 0 && nsteps > 0) {
      if (mesh->use_lo())  // the caller's float state carries no remainder
        FV_CUDA(cudaMemsetAsync(mesh->d_lo, 0, n * sizeof(uint2), s));
      if (cfl > 0.0)
        FV_CUDA(fv::launch_bound(mesh->f64(), U, mesh->d_geom, n, &mesh->d_scal->bmin[0],
                                 &mesh->d_scal->err, s));
      const int64_t chunks = nsteps / kGraphSteps;
      if (chunks > 0) {
        if (!mesh->graph || mesh->g_U != U || mesh->g_scheme != scheme || mesh->g_cfl != cfl ||
            mesh->g_tstop != t_stop || mesh->g_closure != closure ||
            mesh->g_comp != mesh->use_lo())
          capture_graph(mesh, U, cfl, t_stop, scheme, closure);
        for (int64_t k = 0; k < chunks; ++k) FV_CUDA(cudaGraphLaunch(mesh->graph, s));
      }
      const int64_t done = chunks * kGraphSteps;
      enqueue_steps(mesh, U, done, nsteps - done, cfl, t_stop, scheme, s);
      if (scheme == FV_SCHEME_FE && (nsteps % 2) == 1)
        FV_CUDA(cudaMemcpyAsync(U, mesh->d_work, n * mesh->rec_bytes(), cudaMemcpyDeviceToDevice,
                                s));
      mesh->last_t_slot = (int)(nsteps % 2);
    }
    if (t_advanced) read_status(mesh, s, t_advanced, true);
  });
}

int fv_mesh_status(fv_mesh* mesh, void* stream, double* t_advanced) {
  return guarded([&] {
    check_mesh(mesh);
    if (!mesh->stepped || !mesh->d_scal) {
      if (t_advanced) *t_advanced = 0.0;
      return;
    }
    read_status(mesh, as_stream(stream), t_advanced, true);
  });
}

int fv_residual(fv_mesh* mesh, const void* U, void* R, const fv_closure* closure, void* stream) {
  return guarded([&] {
    check_mesh(mesh);
    if (closure) invalid("learned closure is not available in this build");
    if (mesh->h.n == 0) return;
    if (!U || !R) invalid("null state or residual");
    if (U == R) invalid("R must not alias U");
    cudaStream_t s = as_stream(stream);
    ensure_device(mesh, s);
    fv::StepArgs a = base_args(mesh);
    a.U = U;
    a.out = R;
    FV_CUDA(fv::launch_step(mesh->f64(), fv::kModeResidual, a, s));
  });
}

int fv_compute_dt(fv_mesh* mesh, const void* U, double cfl, void* stream, double* dt) {
  return guarded([&] {
    check_mesh(mesh);
    if (!dt) invalid("null dt");
    if (!std::isfinite(cfl) || cfl == 0.0) invalid("cfl must be finite and non-zero");
    if (cfl < 0.0 || mesh->h.n == 0) {
      *dt = cfl < 0.0 ? -cfl : INFINITY;
      return;
    }
    if (!U) invalid("null state");
    cudaStream_t s = as_stream(stream);
    ensure_device(mesh, s);
    fv::LoopScalars* sc = mesh->d_scal;
    FV_CUDA(fv::launch_reset_min(&sc->aux_bmin, &sc->aux_err, s));
    FV_CUDA(fv::launch_bound(mesh->f64(), U, mesh->d_geom, mesh->h.n, &sc->aux_bmin, &sc->aux_err,
                             s));
    FV_CUDA(fv::launch_dt_from_bound(&sc->aux_bmin, cfl, &sc->dt_out, s));
    fv::LoopScalars h{};
    FV_CUDA(cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, s));
    FV_CUDA(cudaStreamSynchronize(s));
    if (h.aux_err) throw fv::Error{FV_ENONFINITE, "state has non-finite values or rho/p <= 0"};
    *dt = h.dt_out;
  });
}

int fv_conserved_totals(fv_mesh* mesh, const void* U, double* out, void* stream) {
  return guarded([&] {
    check_mesh(mesh);
    if (!out) invalid("null out");
    if (mesh->h.n == 0) {
      out[0] = out[1] = out[2] = out[3] = 0.0;
      return;
    }
    if (!U) invalid("null state");
    cudaStream_t s = as_stream(stream);
    ensure_device(mesh, s);
    fv::LoopScalars* sc = mesh->d_scal;
    FV_CUDA(fv::launch_totals(mesh->f64(), U, mesh->d_vol, mesh->h.n, mesh->d_partials,
                              sc->totals, s));
    FV_CUDA(cudaMemcpyAsync(out, sc->totals, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    FV_CUDA(cudaStreamSynchronize(s));
  });
}

}  // extern "C"
