// capi.cu -- the library's C ABI (declared in include/fv.h): handle
// lifetime, host->device upload, the time loop as captured CUDA graphs, and
// status reporting.  Every entry point converts exceptions into a status code
// and a thread-local message.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <iterator>
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
constexpr int kBatchTile = 1024;  // cells per tile of the batched shared-memory shape

}  // namespace

namespace fv {
// Sets this thread's fv_last_error message (for entry points in other files).
int record_error(int code, const std::string& msg) { return set_error(code, msg); }
}  // namespace fv

// Learned dissipation scale: device copies of the packed parameters.
struct fv_closure {
  int device = -1;
  unsigned* d_w1 = nullptr;  // [32 * 4] bfloat16 pairs
  unsigned* d_w2 = nullptr;  // [32 * 16] bfloat16 pairs
  float* d_b = nullptr;      // b1[32] b2[32] w3[32] b3
  float* d_theta = nullptr;  // FP32 staging of theta (kClosureParams)
  float b3 = 0.0f;           // host copy: a kernel argument
  // stamp of the parameters now uploaded, unique in the process: a step
  // graph captured with other parameters (b3 is baked into its launches) or
  // with another closure at the same address is recaptured
  uint64_t version = 0;
  // training scratch: per-block gradient and loss partials, outputs
  int grad_blocks = 0;
  float* d_gpart = nullptr;
  double* d_lpart = nullptr;
  float* d_grad = nullptr;
  double* d_loss = nullptr;

  fv::ClosureParams params() const {
    fv::ClosureParams p;
    p.w1 = d_w1;
    p.w2 = d_w2;
    p.b1 = d_b;
    p.b2 = d_b + 32;
    p.w3 = d_b + 64;
    p.b3 = b3;
    p.tc = false;
    return p;
  }
};

struct fv_mesh {
  fv::HostMesh h;
  int32_t precision = FV_F32;
  double uinf_prim[4] = {1.0, 0.0, 0.0, 1.0};  // rho, u, v, p
  // device side
  int device = -1;
  bool dirty = true;
  int64_t dev_n = -1;
  void* d_nbr = nullptr;   // FP64: int4 per cell; FP32: int2 (nbr1, nbr2)
  void* d_geom = nullptr;  // 8 values per cell (see kernels.h)
  double* d_vol = nullptr;
  void* d_work = nullptr;  // ping-pong partner of the caller's state / RK2 stage
  uint2* d_lo = nullptr;        // FP32 compensated update: remainder of the state
  uint2* d_lo_stage = nullptr;  // ... and of the RK2 stage state
  bool compensated = true;      // FP32 meshes only
  void* user_lo = nullptr;      // caller-owned remainder (fv_mesh_set_remainder)
  int variant = 1;              // step-kernel shape (fv_mesh_autotune / fv_mesh_set_variant)
  // two steps per launch (fv_mesh_set_blocking): tiles and halos on the device
  int blocking = 1;
  int pair_tile = 1024;
  int pair_staged = 0;  // 1: bulk-copy staged two-step kernel
  bool chained = true;  // programmatic dependent launch of the step kernels
  int wave = FV_WAVE_AVERAGE;  // wave speed of the dissipation (fv_mesh_set_wave_speed)
  int closure_engine = FV_CLOSURE_MMA_SYNC;  // fv_mesh_set_closure_engine
  int tiles_built = 0;  // tile size of the arrays below (0: none)
  uint2* d_cell_ln = nullptr;
  int* d_tile_info = nullptr;
  int* d_halo_id = nullptr;
  uint2* d_halo_ln = nullptr;
  int* d_face_off = nullptr;   // shape 7: the faces each tile evaluates once
  uint2* d_face_rec = nullptr;
  int p_e_cap = 0, p_t1_cap = 0;
  // normals from vertex coordinates (fv_mesh_set_geometry): tile nodes
  int geometry = FV_GEOM_STORED;
  bool tiles_vertex = false;  // the tile arrays above carry the vertex layout
  unsigned* d_cell_vl = nullptr;
  int* d_tile_voff = nullptr;
  int2* d_tile_vq = nullptr;
  float* d_inv_vol = nullptr;  // FP32 1/V per cell
  int p_v_cap = 0;
  // learned closure: each face once (owner cell and face, cell across and
  // its face, or a ghost code) and the scale of every cell face
  fv::FaceRec* d_faces = nullptr;
  int64_t n_faces = 0;
  float* d_scale = nullptr;
  unsigned wait_limit = fv::kDefaultWaitLimit;  // bounded device waits (variant 5)
  fv::LoopScalars* d_scal = nullptr;
  double* d_partials = nullptr;
  cudaStream_t cap_stream = nullptr;
  // cached graph of kGraphSteps steps
  cudaGraphExec_t graph = nullptr;
  const void* g_U = nullptr;
  int32_t g_scheme = -1;
  double g_cfl = 0.0, g_tstop = 0.0;
  const fv_closure* g_closure = nullptr;
  uint64_t g_closure_version = 0;
  bool g_comp = false;
  int g_variant = -1;
  int g_blocking = -1, g_tile = -1, g_staged = -1;
  bool g_chained = false;
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

  void free_tiles() {
    dev_free(d_face_off);
    dev_free(d_face_rec);
    dev_free(d_cell_ln);
    dev_free(d_tile_info);
    dev_free(d_halo_id);
    dev_free(d_halo_ln);
    dev_free(d_cell_vl);
    dev_free(d_tile_voff);
    dev_free(d_tile_vq);
    dev_free(d_inv_vol);
    tiles_built = 0;
    tiles_vertex = false;
    p_v_cap = 0;
  }

  bool vertex_tiles() const { return geometry == FV_GEOM_VERTEX; }

  void free_faces() {
    dev_free(d_faces);
    dev_free(d_scale);
    n_faces = 0;
  }

  void free_device() {
    drop_graph();
    free_tiles();
    free_faces();
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

// Tiles and halos of the two-step update, built on the host for the current
// numbering and tile size and copied to the device.
bool tiled_shape(int v) { return v == fv::kTileVariant || v == fv::kFaceTileVariant; }
bool uses_tiles(const fv_mesh* m) { return m->blocking == 2 || tiled_shape(m->variant); }

// The faces each tile evaluates once (shape 7), uploaded when that shape
// first runs on the current tiles.
void upload_tile_faces(fv_mesh* m, const fv::PairTiles& L, cudaStream_t s) {
  FV_CUDA(cudaMalloc((void**)&m->d_face_off, L.face_off.size() * sizeof(int32_t)));
  FV_CUDA(cudaMalloc((void**)&m->d_face_rec, std::max<size_t>(L.face_rec.size(), 2) *
                                                  sizeof(uint32_t)));
  FV_CUDA(cudaMemcpyAsync(m->d_face_off, L.face_off.data(), L.face_off.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice, s));
  FV_CUDA(cudaMemcpyAsync(m->d_face_rec, L.face_rec.data(), L.face_rec.size() * sizeof(uint32_t),
                          cudaMemcpyHostToDevice, s));
  FV_CUDA(cudaStreamSynchronize(s));  // L is a staging buffer
}

void ensure_tiles(fv_mesh* m, cudaStream_t s) {
  if (!uses_tiles(m) || m->h.n == 0) return;
  if (m->tiles_built == m->pair_tile && m->tiles_vertex == m->vertex_tiles()) {
    if (m->variant == fv::kFaceTileVariant && !m->d_face_rec) {
      m->drop_graph();
      upload_tile_faces(m, fv::build_pair_tiles(m->h, m->pair_tile), s);
    }
    return;
  }
  m->free_tiles();
  m->drop_graph();
  fv::PairTiles L = fv::build_pair_tiles(m->h, m->pair_tile);
  if (m->variant == fv::kFaceTileVariant && !m->vertex_tiles()) upload_tile_faces(m, L, s);
  fv::TileVertices V;
  if (m->vertex_tiles()) {
    V = fv::build_tile_vertices(m->h, m->pair_tile);
    for (int64_t c = 0; c < m->h.n; ++c)  // node 0 replaces the reverse-face bits
      L.cell_ln[2 * c + 1] = (L.cell_ln[2 * c + 1] & 0xFFFFu) | ((uint32_t)V.v0[c] << 16);
    const size_t ncells = (size_t)m->h.n;
    FV_CUDA(cudaMalloc((void**)&m->d_cell_vl, ncells * sizeof(unsigned)));
    FV_CUDA(cudaMalloc((void**)&m->d_inv_vol, ncells * sizeof(float)));
    V.inv_vol.resize(ncells);  // the FP32 1/V of the geometry records
    for (size_t c = 0; c < ncells; ++c) V.inv_vol[c] = (float)(1.0 / m->h.vol[c]);
    FV_CUDA(cudaMemcpyAsync(m->d_inv_vol, V.inv_vol.data(), ncells * sizeof(float),
                            cudaMemcpyHostToDevice, s));
    FV_CUDA(cudaMalloc((void**)&m->d_tile_voff, V.voff.size() * sizeof(int32_t)));
    FV_CUDA(cudaMalloc((void**)&m->d_tile_vq, std::max<size_t>(V.vq.size(), 2) * sizeof(int32_t)));
    FV_CUDA(cudaMemcpyAsync(m->d_cell_vl, V.cell_vl.data(), ncells * sizeof(unsigned),
                            cudaMemcpyHostToDevice, s));
    FV_CUDA(cudaMemcpyAsync(m->d_tile_voff, V.voff.data(), V.voff.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));
    FV_CUDA(cudaMemcpyAsync(m->d_tile_vq, V.vq.data(), V.vq.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));
  }
  // whole 256-cell tiles: the staged kernel copies an even number of records
  const size_t ncells = (size_t)((m->h.n + fv::kPadCells - 1) / fv::kPadCells * fv::kPadCells);
  FV_CUDA(cudaMalloc((void**)&m->d_cell_ln, ncells * sizeof(uint2)));
  FV_CUDA(cudaMalloc((void**)&m->d_tile_info, L.tile_info.size() * sizeof(int32_t)));
  const size_t nh = std::max<size_t>(L.halo_id.size(), 1);
  FV_CUDA(cudaMalloc((void**)&m->d_halo_id, nh * sizeof(int32_t)));
  FV_CUDA(cudaMalloc((void**)&m->d_halo_ln, nh * sizeof(uint2)));
  FV_CUDA(cudaMemcpyAsync(m->d_cell_ln, L.cell_ln.data(), L.cell_ln.size() * sizeof(uint32_t),
                          cudaMemcpyHostToDevice, s));
  FV_CUDA(cudaMemcpyAsync(m->d_tile_info, L.tile_info.data(), L.tile_info.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice, s));
  if (!L.halo_id.empty()) {
    FV_CUDA(cudaMemcpyAsync(m->d_halo_id, L.halo_id.data(), L.halo_id.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));
    FV_CUDA(cudaMemcpyAsync(m->d_halo_ln, L.halo_ln.data(), L.halo_ln.size() * sizeof(uint32_t),
                            cudaMemcpyHostToDevice, s));
  }
  FV_CUDA(cudaStreamSynchronize(s));  // L is a local staging buffer
  m->p_e_cap = L.e_cap;
  m->p_t1_cap = L.t1_cap;
  m->p_v_cap = V.v_cap;
  m->tiles_vertex = m->vertex_tiles();
  m->tiles_built = m->pair_tile;
}

// Shared memory of the one-step tile kernel of this mesh.
size_t tile_smem(const fv_mesh* m) {
  return fv::tile_smem_bytes(m->f64(), m->p_t1_cap, m->tiles_vertex ? m->p_v_cap : 0);
}

// ... and of the step kernel of the mesh's tiled shape (6 or 7)
size_t step_tile_smem(const fv_mesh* m) {
  return m->variant == fv::kFaceTileVariant
             ? fv::tile_faces_smem_bytes(m->f64(), m->p_t1_cap, m->tiles_built)
             : tile_smem(m);
}

// Shared memory a tiled kernel of this mesh needs, checked against the device.
void check_tile_smem(const fv_mesh* m, size_t smem) {
  int dev = 0, optin = 0;
  FV_CUDA(cudaGetDevice(&dev));
  FV_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > (size_t)optin)
    invalid("a tile with its halos needs " + std::to_string(smem) + " bytes of shared memory (" +
            std::to_string(optin) + " available); renumber the cells with a compact order "
            "(Hilbert) or use smaller tiles");
}

// Tile sizes the autotuner times for the one-step tile shape: the standard
// ones, and on a mesh of a few waves of resident blocks the sizes that fill
// whole waves (w waves of b blocks per SM), which avoid a last, partly
// filled wave.
std::vector<int> tile_candidates(int64_t n) {
  // small tiles suit shape 7, whose face records take shared memory
  std::vector<int> t = {256, 384};
  t.insert(t.end(), std::begin(fv::kPairTiles), std::end(fv::kPairTiles));
  int dev = 0, sms = 0;
  FV_CUDA(cudaGetDevice(&dev));
  FV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  for (int b : {5, 4, 2})  // resident blocks per SM of the FP32 / FP64 shapes
    for (int w = 1; w <= 3; ++w) {
      const int64_t slots = (int64_t)w * b * sms;
      const int64_t c = ((n + slots - 1) / slots + 31) / 32 * 32;
      if (c >= 64 && c <= fv::kMaxTileCells && std::find(t.begin(), t.end(), (int)c) == t.end())
        t.push_back((int)c);
    }
  return t;
}

size_t pair_smem(const fv_mesh* m) {
  return fv::pair_smem_bytes(m->p_e_cap, m->p_t1_cap, m->tiles_built, m->pair_staged != 0);
}

void ensure_device(fv_mesh* m, cudaStream_t s) {
  int dev = 0;
  FV_CUDA(cudaGetDevice(&dev));
  if (m->device >= 0 && m->device != dev && m->dev_n >= 0)
    invalid("mesh was uploaded to device " + std::to_string(m->device) +
            " but the current device is " + std::to_string(dev));
  if (!m->dirty && m->dev_n == m->h.n) {
    ensure_tiles(m, s);
    return;
  }
  m->free_tiles();
  m->free_faces();
  const int64_t n = m->h.n;
  if (m->dev_n != n) {
    m->free_device();
    // whole tiles: the TMA-staged step copies whole tiles of these arrays
    const size_t nn = (size_t)((std::max<int64_t>(n, 1) + fv::kPadCells - 1) / fv::kPadCells *
                               fv::kPadCells);
    FV_CUDA(cudaMalloc(&m->d_nbr, nn * (m->f64() ? sizeof(int4) : sizeof(int2))));
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
  if (n > 0) {
    fv::DeviceLayout lay = fv::pack_layout(m->h.nbr.data(), m->h.nrm.data(), m->h.vol.data(),
                                           m->h.inradius.data(), n, 0, m->f64());
    FV_CUDA(cudaMemcpyAsync(m->d_nbr, lay.nbr.data(), lay.nbr.size(), cudaMemcpyHostToDevice, s));
    FV_CUDA(cudaMemcpyAsync(m->d_geom, lay.geom.data(), lay.geom.size(), cudaMemcpyHostToDevice,
                            s));
    FV_CUDA(cudaMemcpyAsync(m->d_vol, m->h.vol.data(), n * sizeof(double), cudaMemcpyHostToDevice,
                            s));
    FV_CUDA(cudaStreamSynchronize(s));  // lay is a local staging buffer
  }
  FV_CUDA(cudaStreamSynchronize(s));
  m->device = dev;
  m->dirty = false;
  ensure_tiles(m, s);
}

// The faces of the mesh, each once, for the learned closure's scale pass:
// (4 a + ka, 4 b + kb) for the face ka of cell a whose other side is face kb
// of cell b (a <= b; a cell may border itself across a periodic seam), and
// (4 a + ka, ghost code) for a boundary face, with face ka's normal as the
// FP32 geometry record rounds it.  The two sides of a face are matched by
// neighbour id and exactly opposite normals.
std::vector<fv::FaceRec> closure_faces(const fv::HostMesh& h) {
  std::vector<fv::FaceRec> f;
  f.reserve((size_t)(2 * h.n));
  auto rec = [&](int64_t c, int k, int b) {
    return fv::FaceRec{(int)(4 * c + k), b, (float)h.nrm[6 * c + 2 * k],
                       (float)h.nrm[6 * c + 2 * k + 1]};
  };
  for (int64_t c = 0; c < h.n; ++c)
    for (int k = 0; k < 3; ++k) {
      const int32_t m = h.nbr[3 * c + k];
      if (m < 0) {
        f.push_back(rec(c, k, m));
        continue;
      }
      if (m < c) continue;
      int km = -1;
      for (int q = 0; q < 3; ++q)
        if (h.nbr[3 * (int64_t)m + q] == (int32_t)c && !(m == c && q == k) &&
            h.nrm[6 * (int64_t)m + 2 * q] == -h.nrm[6 * c + 2 * k] &&
            h.nrm[6 * (int64_t)m + 2 * q + 1] == -h.nrm[6 * c + 2 * k + 1])
          km = q;
      if (km < 0) invalid("closure faces: the two sides of a face do not match");
      if (m == c && km < k) continue;  // a self-face is listed from its lower index
      f.push_back(rec(c, k, (int)(4 * (int64_t)m + km)));
    }
  return f;
}

void ensure_faces(fv_mesh* m, cudaStream_t s) {
  if (m->d_faces) return;
  if (4 * m->h.n > INT32_MAX) invalid("the learned closure takes meshes below 2^29 cells");
  const std::vector<fv::FaceRec> f = closure_faces(m->h);
  FV_CUDA(cudaMalloc((void**)&m->d_faces, std::max<size_t>(f.size(), 1) * sizeof(fv::FaceRec)));
  FV_CUDA(cudaMalloc((void**)&m->d_scale, std::max<int64_t>(3 * m->h.n, 1) * sizeof(float)));
  FV_CUDA(cudaMemcpyAsync(m->d_faces, f.data(), f.size() * sizeof(fv::FaceRec),
                          cudaMemcpyHostToDevice, s));
  FV_CUDA(cudaStreamSynchronize(s));  // f is a local staging buffer
  m->n_faces = (int64_t)f.size();
}

fv::StepArgs base_args(const fv_mesh* m) {
  fv::StepArgs a{};
  a.nbr = m->d_nbr;
  a.geom = m->d_geom;
  a.n = m->h.n;
  m->uinf_conserved(a.uinf);
  for (int q = 0; q < 4; ++q) a.uinf_f[q] = (float)a.uinf[q];
  a.err = &m->d_scal->err;
  a.wait_limit = m->wait_limit;
  a.drain_limit = fv::kDefaultWaitLimit;
  a.chained = m->chained;
  a.wave = m->wave == FV_WAVE_MAX ? fv::kWaveMax : fv::kWaveAverage;
  if (m->tiles_built) {
    a.cell_ln = m->d_cell_ln;
    a.tile_info = m->d_tile_info;
    a.halo_id = m->d_halo_id;
    a.tile = m->tiles_built;
    a.t1_cap = m->p_t1_cap;
    a.tile_face_off = m->d_face_off;
    a.tile_face = m->d_face_rec;
    if (m->tiles_vertex) {
      a.cell_vl = m->d_cell_vl;
      a.tile_voff = m->d_tile_voff;
      a.tile_vq = m->d_tile_vq;
      a.inv_vol = m->d_inv_vol;
      a.v_cap = m->p_v_cap;
      a.vscale = (float)std::ldexp(1.0, m->h.grid_e);
    }
  }
  return a;
}

// The closure's parameters with the mesh's tensor-core engine.
fv::ClosureParams closure_params(const fv_mesh* m, const fv_closure* cl) {
  fv::ClosureParams p = cl->params();
  p.tc = m->closure_engine == FV_CLOSURE_TCGEN05;
  return p;
}

cudaError_t launch_mode(const fv_mesh* m, int mode, const fv::StepArgs& a, const fv_closure* cl,
                        cudaStream_t s) {
  if (cl && m->variant == fv::kFaceTileVariant)  // one launch on the tiles of shape 7
    return fv::launch_step_closure_tile(mode, a, closure_params(m, cl), s);
  if (cl) {
    // the scales of the state the stage evaluates, then the scaled step
    cudaError_t e =
        fv::launch_face_scales(a, m->d_faces, m->n_faces, closure_params(m, cl), m->d_scale, s);
    if (e != cudaSuccess) return e;
    return fv::launch_step_scaled(mode, a, m->d_scale, s);
  }
  return fv::launch_step(m->f64(), mode, m->variant, a, s);
}

// Enqueues steps j0 .. j0+count-1 of a loop on stream s.
void enqueue_steps(fv_mesh* m, void* U, int64_t j0, int64_t count, double cfl, double t_stop,
                   int32_t scheme, cudaStream_t s, const fv_closure* cl = nullptr,
                   bool lo_alt = false) {
  fv::LoopScalars* sc = m->d_scal;
  if (!cl && tiled_shape(m->variant) && count > 0) check_tile_smem(m, step_tile_smem(m));
  if (cl && m->variant == fv::kFaceTileVariant && count > 0) {
    if (m->tiles_built > 1024) invalid("the learned closure on tiles takes tiles of up to 1024 cells");
    check_tile_smem(m, fv::closure_tile_smem_bytes(m->p_t1_cap, m->tiles_built,
                                                   m->closure_engine == FV_CLOSURE_TCGEN05));
  }
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
      // lo_alt: after an odd number of two-step launches the remainder of the
      // state is in the second buffer (forward Euler only)
      a.lo = lo_alt ? m->d_lo_stage : m->d_lo;
      a.lo_stage = m->d_lo_stage;
    }
    if (scheme == FV_SCHEME_FE) {
      const bool even = (j % 2) == 0;
      a.U = even ? U : m->d_work;
      a.out = even ? m->d_work : U;
      FV_CUDA(launch_mode(m, fv::kModeFE, a, cl, s));
    } else {
      a.U = U;
      a.out = m->d_work;
      FV_CUDA(launch_mode(m, fv::kModeRK2a, a, cl, s));
      a.U = m->d_work;
      a.Ubase = U;
      a.out = U;
      FV_CUDA(launch_mode(m, fv::kModeRK2b, a, cl, s));
    }
  }
}

// Enqueues two-step launches j0 .. j0+count-1 (forward Euler).  Launch j reads
// the state and remainder from U and d_lo when j is even, from the work
// buffers when it is odd, and writes the others; the scalar slots rotate per
// launch as they do per step.
void enqueue_pairs(fv_mesh* m, void* U, int64_t j0, int64_t count, double cfl, double t_stop,
                   cudaStream_t s) {
  fv::LoopScalars* sc = m->d_scal;
  if (count > 0) check_tile_smem(m, pair_smem(m));
  for (int64_t j = j0; j < j0 + count; ++j) {
    const bool even = (j % 2) == 0;
    fv::PairArgs a{};
    a.U = static_cast<const float4*>(even ? U : m->d_work);
    a.out = static_cast<float4*>(even ? m->d_work : U);
    if (m->use_lo()) {
      a.lo_in = even ? m->d_lo : m->d_lo_stage;
      a.lo_out = even ? m->d_lo_stage : m->d_lo;
    }
    a.geom = static_cast<const float4*>(m->d_geom);
    a.cell_ln = m->d_cell_ln;
    a.tile_info = m->d_tile_info;
    a.halo_id = m->d_halo_id;
    a.halo_ln = m->d_halo_ln;
    a.n = m->h.n;
    a.tile = m->tiles_built;
    a.e_cap = m->p_e_cap;
    a.t1_cap = m->p_t1_cap;
    double ui[4];
    m->uinf_conserved(ui);
    for (int q = 0; q < 4; ++q) a.uinf[q] = (float)ui[q];
    a.bmin_read = &sc->bmin[j % 3];
    a.bmin_write = &sc->bmin[(j + 1) % 3];
    a.bmin_reset = &sc->bmin[(j + 2) % 3];
    a.t_read = &sc->t[j % 2];
    a.t_write = &sc->t[(j + 1) % 2];
    a.cfl = cfl;
    a.t_stop = t_stop;
    a.err = &sc->err;
    a.wait_limit = m->wait_limit;
    a.drain_limit = fv::kDefaultWaitLimit;
    a.chained = m->chained;
    FV_CUDA(fv::launch_step_pair(a, m->pair_staged, s));
  }
}

// Steps of one time loop: whole launches [j0, j0 + launches) of the mesh's
// kind (one step each, or two with blocking).
void enqueue_launches(fv_mesh* m, void* U, int64_t j0, int64_t launches, double cfl,
                      double t_stop, int32_t scheme, cudaStream_t s, const fv_closure* cl) {
  if (m->blocking == 2)
    enqueue_pairs(m, U, j0, launches, cfl, t_stop, s);
  else
    enqueue_steps(m, U, j0, launches, cfl, t_stop, scheme, s, cl);
}

void capture_graph(fv_mesh* m, void* U, double cfl, double t_stop, int32_t scheme,
                   const fv_closure* cl) {
  m->drop_graph();
  cudaGraph_t g = nullptr;
  FV_CUDA(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
  try {
    enqueue_launches(m, U, 0, kGraphSteps / m->blocking, cfl, t_stop, scheme, m->cap_stream, cl);
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
  m->g_closure_version = cl ? cl->version : 0;
  m->g_comp = m->use_lo();
  m->g_variant = m->variant;
  m->g_blocking = m->blocking;
  m->g_tile = m->tiles_built;
  m->g_staged = m->pair_staged;
  m->g_chained = m->chained;
}

void read_status(fv_mesh* m, cudaStream_t s, double* t_adv, bool check) {
  fv::LoopScalars h{};
  FV_CUDA(cudaMemcpyAsync(&h, m->d_scal, sizeof h, cudaMemcpyDeviceToHost, s));
  FV_CUDA(cudaStreamSynchronize(s));
  if (t_adv) *t_adv = h.t[m->last_t_slot];
  if (check && (h.err & 8))
    throw fv::Error{FV_EINDEX, "a neighbour, halo or node index was outside its array "
                               "(bounds-checked build); the state is not valid"};
  if (check && (h.err & 4))
    throw fv::Error{FV_ESTATE, "a bounded device wait gave up and the copies in flight did not "
                               "drain either; destroy the mesh"};
  if (check && (h.err & 2))
    throw fv::Error{FV_ETIMEOUT, "a bounded device wait gave up; the state is not valid"};
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

int32_t fv_index_checks(void) {
#ifdef FV_DEBUG
  return 1;
#else
  return 0;
#endif
}

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
      case FV_ORDER_AM1: perm = fv::order_am1(mesh->h); break;
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

int fv_mesh_set_remainder(fv_mesh* mesh, void* lo) {
  return guarded([&] {
    check_mesh(mesh);
    if (lo && mesh->f64()) invalid("FV_F64 meshes have no remainder");
    mesh->user_lo = lo;
  });
}

int fv_mesh_set_variant(fv_mesh* mesh, int32_t variant) {
  return guarded([&] {
    check_mesh(mesh);
    if (variant < 0 || variant >= fv::kStepVariants) invalid("unknown step-kernel variant");
    if (variant == fv::kFaceTileVariant && mesh->vertex_tiles())
      invalid("normals from node coordinates run the tile shape 6");
    mesh->variant = variant;
    mesh->drop_graph();
  });
}

int fv_mesh_set_blocking(fv_mesh* mesh, int32_t steps_per_launch, int32_t tile_cells,
                         int32_t staged) {
  return guarded([&] {
    check_mesh(mesh);
    if (steps_per_launch != 1 && steps_per_launch != 2) invalid("steps_per_launch must be 1 or 2");
    if (staged != 0 && staged != 1) invalid("staged must be 0 or 1");
    if (tile_cells == 0) tile_cells = 1024;
    bool known = false;
    for (int t : fv::kPairTiles) known = known || t == tile_cells;
    if (steps_per_launch == 2 && !known)
      invalid("with two steps per launch tile_cells must be 0, 512, 768, 1024 or 2048");
    if (tile_cells < 32 || tile_cells > fv::kMaxTileCells)
      invalid("tile_cells must be 0 or 32 .. 2048");
    if (staged && tile_cells != 512 && tile_cells != 1024)
      invalid("the staged kernel takes tiles of 512 or 1024 cells");
    if (steps_per_launch == 2 && mesh->f64())
      invalid("two steps per launch are built for FV_F32 meshes (the FP64 step is bound by "
              "arithmetic, not by memory)");
    if (staged != mesh->pair_staged) mesh->tiles_built = 0;  // shared-memory check differs
    mesh->blocking = steps_per_launch;
    mesh->pair_tile = tile_cells;
    mesh->pair_staged = staged;
    mesh->drop_graph();
  });
}

int fv_mesh_get_tiling(const fv_mesh* mesh, int32_t* variant, int32_t* tile_cells) {
  return guarded([&] {
    check_mesh(mesh);
    if (variant) *variant = mesh->variant;
    if (tile_cells) *tile_cells = mesh->pair_tile;
  });
}

int fv_mesh_tile_halo(const fv_mesh* mesh, int32_t tile_cells, int64_t tile, int32_t* halo_ids,
                      int64_t capacity, int64_t* n_first, int64_t* n_second) {
  return guarded([&] {
    check_mesh(mesh);
    const fv::PairTiles L = fv::build_pair_tiles(mesh->h, tile_cells);
    if (tile < 0 || tile >= L.n_tiles) invalid("tile index out of range");
    const int64_t hs = L.tile_info[2 * tile], h1 = L.tile_info[2 * tile + 1];
    const int64_t h12 = L.tile_info[2 * tile + 2] - hs;
    if (n_first) *n_first = h1;
    if (n_second) *n_second = h12 - h1;
    if (halo_ids) {
      if (capacity < h12) invalid("halo_ids capacity too small");
      std::memcpy(halo_ids, L.halo_id.data() + hs, h12 * sizeof(int32_t));
    }
  });
}

int fv_mesh_tile_nodes(const fv_mesh* mesh, int32_t tile_cells, int64_t tile, int32_t* grid_xy,
                       int64_t capacity, int64_t* n_nodes, uint16_t* cell_local) {
  return guarded([&] {
    check_mesh(mesh);
    if (!mesh->h.snapped()) invalid("tile nodes exist only on a mesh with vertex geometry");
    const fv::TileVertices V = fv::build_tile_vertices(mesh->h, tile_cells);
    const int64_t n_tiles = (int64_t)V.voff.size() - 1;
    if (tile < 0 || tile >= n_tiles) invalid("tile index out of range");
    const int64_t v0 = V.voff[tile], nb = V.voff[tile + 1] - v0;
    if (n_nodes) *n_nodes = nb;
    if (grid_xy) {
      if (capacity < nb) invalid("grid_xy capacity too small");
      std::memcpy(grid_xy, V.vq.data() + 2 * v0, 2 * nb * sizeof(int32_t));
    }
    if (cell_local) {
      const int64_t c0 = tile * (int64_t)tile_cells;
      const int64_t c1 = std::min<int64_t>(c0 + tile_cells, mesh->h.n);
      for (int64_t c = c0; c < c1; ++c) {
        cell_local[3 * (c - c0)] = V.v0[c];
        cell_local[3 * (c - c0) + 1] = (uint16_t)(V.cell_vl[c] & 0xffffu);
        cell_local[3 * (c - c0) + 2] = (uint16_t)(V.cell_vl[c] >> 16);
      }
    }
  });
}

int fv_mesh_set_geometry(fv_mesh* mesh, int32_t form) {
  return guarded([&] {
    check_mesh(mesh);
    if (form == FV_GEOM_STORED) {
      mesh->geometry = form;
    } else if (form == FV_GEOM_VERTEX) {
      if (mesh->f64())
        invalid("vertex geometry is built for FV_F32 meshes (the FP64 step is bound by "
                "arithmetic, not by memory)");
      if (!mesh->h.snapped()) {
        fv::snap_to_vertex_grid(mesh->h);  // throws before changing the mesh
        mesh->dirty = true;                // geometry records of the snapped mesh
      }
      mesh->geometry = form;
      mesh->variant = fv::kTileVariant;
    } else {
      invalid("unknown geometry form");
    }
    mesh->drop_graph();
  });
}

int fv_mesh_nodes(const fv_mesh* mesh, int64_t* n_nodes, double* xy, int32_t* grid_exponent) {
  return guarded([&] {
    check_mesh(mesh);
    if (n_nodes) *n_nodes = (int64_t)mesh->h.node_xy.size() / 2;
    if (xy) std::memcpy(xy, mesh->h.node_xy.data(), mesh->h.node_xy.size() * sizeof(double));
    if (grid_exponent) *grid_exponent = mesh->h.snapped() ? mesh->h.grid_e : INT32_MIN;
  });
}

int fv_mesh_set_wave_speed(fv_mesh* mesh, int32_t mode) {
  return guarded([&] {
    check_mesh(mesh);
    if (mode != FV_WAVE_AVERAGE && mode != FV_WAVE_MAX) invalid("unknown wave-speed mode");
    mesh->wave = mode;
    mesh->drop_graph();
  });
}

int fv_mesh_set_closure_engine(fv_mesh* mesh, int32_t engine) {
  return guarded([&] {
    check_mesh(mesh);
    if (engine != FV_CLOSURE_MMA_SYNC && engine != FV_CLOSURE_TCGEN05)
      invalid("unknown closure engine");
    mesh->closure_engine = engine;
    mesh->drop_graph();
  });
}

int fv_mesh_set_launch_chaining(fv_mesh* mesh, int32_t enable) {
  return guarded([&] {
    check_mesh(mesh);
    mesh->chained = enable != 0;
    mesh->drop_graph();
  });
}

int fv_mesh_set_wait_limit(fv_mesh* mesh, uint32_t polls) {
  return guarded([&] {
    check_mesh(mesh);
    mesh->wait_limit = polls;
    mesh->drop_graph();
  });
}

int fv_mesh_autotune(fv_mesh* mesh, const void* U, int32_t scheme, void* stream, int32_t* best,
                     double* us_per_step) {
  return guarded([&] {
    check_mesh(mesh);
    if (scheme != FV_SCHEME_FE && scheme != FV_SCHEME_RK2) invalid("unknown scheme");
    const int64_t n = mesh->h.n;
    if (n == 0) {
      if (best) *best = mesh->variant;
      return;
    }
    if (!U) invalid("null state");
    cudaStream_t s = as_stream(stream);
    ensure_device(mesh, s);
    void* tmp = nullptr;
    FV_CUDA(cudaMalloc(&tmp, n * mesh->rec_bytes()));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double times[fv::kStepVariants];
    const int keep = mesh->variant, keep_tile = mesh->pair_tile;
    int best_tile[fv::kStepVariants];
    for (int v = 0; v < fv::kStepVariants; ++v) best_tile[v] = keep_tile;
    try {
      FV_CUDA(cudaEventCreate(&e0));
      FV_CUDA(cudaEventCreate(&e1));
      // a negligible fixed dt: the kernels do their full work, the state barely moves
      const double cfl = -1e-30;
      const int64_t steps = std::max<int64_t>(8, std::min<int64_t>(64, (int64_t)(4e7 / (double)n)));
      auto time_shape = [&]() {
        FV_CUDA(cudaMemcpyAsync(tmp, U, n * mesh->rec_bytes(), cudaMemcpyDeviceToDevice, s));
        if (mesh->use_lo()) FV_CUDA(cudaMemsetAsync(mesh->d_lo, 0, n * sizeof(uint2), s));
        FV_CUDA(fv::launch_init_scalars(mesh->d_scal, s));
        enqueue_steps(mesh, tmp, 0, 2, cfl, 0.0, scheme, s);  // warm-up
        FV_CUDA(cudaEventRecord(e0, s));
        enqueue_steps(mesh, tmp, 2, steps, cfl, 0.0, scheme, s);
        FV_CUDA(cudaEventRecord(e1, s));
        FV_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        FV_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return 1e3 * ms / (double)steps;
      };
      for (int v = 0; v < fv::kStepVariants; ++v) {
        mesh->variant = v;
        if (!tiled_shape(v)) {
          // vertex geometry is a layout of the tile shape
          times[v] = mesh->vertex_tiles() ? INFINITY : time_shape();
          continue;
        }
        // the tiled shapes at each tile size; tiles that do not fit (a
        // long-band order) leave that size out
        times[v] = INFINITY;
        if (v == fv::kFaceTileVariant && mesh->vertex_tiles()) continue;
        for (int tile : tile_candidates(n)) {
          mesh->pair_tile = tile;
          try {
            ensure_tiles(mesh, s);
            check_tile_smem(mesh, step_tile_smem(mesh));
          } catch (const fv::Error&) {
            continue;
          }
          const double us = time_shape();
          if (us < times[v]) {
            times[v] = us;
            best_tile[v] = tile;
          }
        }
      }
    } catch (...) {
      mesh->variant = keep;
      mesh->pair_tile = keep_tile;
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      cudaFree(tmp);
      throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    FV_CUDA(cudaStreamSynchronize(s));
    cudaFree(tmp);
    int b = mesh->vertex_tiles() ? fv::kTileVariant : 0;
    for (int v = 0; v < fv::kStepVariants; ++v)
      if (times[v] < times[b]) b = v;
    mesh->variant = b;
    // the tile size of the tiled shapes: the fastest for shape 6 when it wins
    // (two steps per launch keep their own tile size: the two-step kernel
    // takes the standard sizes only)
    mesh->pair_tile = tiled_shape(b) && mesh->blocking == 1 ? best_tile[b] : keep_tile;
    mesh->drop_graph();
    if (best) *best = b;
    if (us_per_step)
      for (int v = 0; v < fv::kStepVariants; ++v) us_per_step[v] = times[v];
  });
}

int fv_partition_sizes(const fv_mesh* mesh, int32_t nparts, int32_t part, int64_t* n_owned,
                       int64_t* n_halo) {
  return guarded([&] {
    check_mesh(mesh);
    const fv::LocalPart lp = fv::build_local_part(mesh->h, nparts, part);
    if (n_owned) *n_owned = lp.n_owned;
    if (n_halo) *n_halo = (int64_t)lp.global.size() - lp.n_owned;
  });
}

int fv_partition_local(const fv_mesh* mesh, int32_t nparts, int32_t part, int64_t* global_ids,
                       int32_t* halo_owner, int32_t* nbr, double* normals, double* area) {
  return guarded([&] {
    check_mesh(mesh);
    const fv::LocalPart lp = fv::build_local_part(mesh->h, nparts, part);
    const int64_t nh = (int64_t)lp.global.size() - lp.n_owned;
    if (global_ids) std::memcpy(global_ids, lp.global.data(), lp.global.size() * sizeof(int64_t));
    if (halo_owner) std::memcpy(halo_owner, lp.halo_owner.data(), nh * sizeof(int32_t));
    if (nbr) std::memcpy(nbr, lp.nbr.data(), lp.nbr.size() * sizeof(int32_t));
    if (normals) std::memcpy(normals, lp.nrm.data(), lp.nrm.size() * sizeof(double));
    if (area) std::memcpy(area, lp.vol.data(), lp.vol.size() * sizeof(double));
  });
}

int fv_mesh_upload(fv_mesh* mesh, void* stream) {
  return guarded([&] {
    check_mesh(mesh);
    ensure_device(mesh, as_stream(stream));
  });
}

int fv_mesh_debug_set_index(fv_mesh* mesh, int32_t table, int64_t cell, int32_t slot,
                            int32_t value, void* stream) {
  return guarded([&] {
    check_mesh(mesh);
    if (!fv_index_checks()) invalid("only bounds-checked builds (FV_DEBUG) take this call");
    if (cell < 0 || cell >= mesh->h.n || slot < 0 || slot > 2) invalid("cell or slot out of range");
    cudaStream_t s = as_stream(stream);
    ensure_device(mesh, s);
    if (table == 0) {
      // global neighbour ids: FP32 keeps face 0's in the geometry record
      if (mesh->f64()) {
        int* p = static_cast<int*>(mesh->d_nbr) + 4 * cell + slot;
        FV_CUDA(cudaMemcpyAsync(p, &value, sizeof value, cudaMemcpyHostToDevice, s));
      } else if (slot == 0) {
        float* p = static_cast<float*>(mesh->d_geom) + 8 * cell + 7;
        FV_CUDA(cudaMemcpyAsync(p, &value, sizeof value, cudaMemcpyHostToDevice, s));
      } else {
        int* p = static_cast<int*>(mesh->d_nbr) + 2 * cell + (slot - 1);
        FV_CUDA(cudaMemcpyAsync(p, &value, sizeof value, cudaMemcpyHostToDevice, s));
      }
    } else if (table == 1) {
      if (!mesh->tiles_built) invalid("no tiles built: step a tiled shape first");
      if (value < 0 || value > 0xFFFF) invalid("tile-local ids are 16-bit");
      uint2 ln{};
      FV_CUDA(cudaMemcpyAsync(&ln, mesh->d_cell_ln + cell, sizeof ln, cudaMemcpyDeviceToHost, s));
      FV_CUDA(cudaStreamSynchronize(s));
      unsigned* w = slot < 2 ? &ln.x : &ln.y;
      const int sh = slot == 1 ? 16 : 0;
      *w = (*w & ~(0xFFFFu << sh)) | ((unsigned)value << sh);
      FV_CUDA(cudaMemcpyAsync(mesh->d_cell_ln + cell, &ln, sizeof ln, cudaMemcpyHostToDevice, s));
    } else {
      invalid("table must be 0 (neighbour ids) or 1 (tile-local ids)");
    }
    FV_CUDA(cudaStreamSynchronize(s));
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
    if (closure && mesh->f64()) invalid("the learned closure runs on FV_F32 meshes only");
    if (mesh->blocking == 2 && (scheme != FV_SCHEME_FE || closure))
      invalid("two steps per launch apply to forward Euler without a closure");
    if (mesh->wave != FV_WAVE_AVERAGE && (closure || mesh->blocking == 2))
      invalid("the maximum wave speed runs without a closure, one step per launch");
    if (!U && nsteps > 0 && mesh->h.n > 0) invalid("null state");
    cudaStream_t s = as_stream(stream);
    ensure_device(mesh, s);
    if (closure) ensure_faces(mesh, s);
    const int64_t n = mesh->h.n;
    FV_CUDA(fv::launch_init_scalars(mesh->d_scal, s));
    mesh->last_t_slot = 0;
    mesh->stepped = true;
    if (n > 0 && nsteps > 0) {
      if (mesh->use_lo()) {
        if (mesh->user_lo)  // the remainder the caller kept from the last call
          FV_CUDA(cudaMemcpyAsync(mesh->d_lo, mesh->user_lo, n * sizeof(uint2),
                                  cudaMemcpyDeviceToDevice, s));
        else  // the caller's float state carries no remainder
          FV_CUDA(cudaMemsetAsync(mesh->d_lo, 0, n * sizeof(uint2), s));
      }
      if (cfl > 0.0)
        FV_CUDA(fv::launch_bound(mesh->f64(), U, mesh->d_geom, n, &mesh->d_scal->bmin[0],
                                 &mesh->d_scal->err, s));
      const int64_t chunks = nsteps / kGraphSteps;
      if (chunks > 0) {
        if (!mesh->graph || mesh->g_U != U || mesh->g_scheme != scheme || mesh->g_cfl != cfl ||
            mesh->g_tstop != t_stop || mesh->g_closure != closure ||
            mesh->g_closure_version != (closure ? closure->version : 0) ||
            mesh->g_comp != mesh->use_lo() || mesh->g_variant != mesh->variant ||
            mesh->g_blocking != mesh->blocking || mesh->g_tile != mesh->tiles_built ||
            mesh->g_staged != mesh->pair_staged || mesh->g_chained != mesh->chained)
          capture_graph(mesh, U, cfl, t_stop, scheme, closure);
        for (int64_t k = 0; k < chunks; ++k) FV_CUDA(cudaGraphLaunch(mesh->graph, s));
      }
      // a graph holds an even number of launches (and a multiple of 3), so the
      // launches after it start from the buffers and slots of launch 0
      const int64_t rest = nsteps - chunks * kGraphSteps;
      const int64_t tail = rest / mesh->blocking;
      enqueue_launches(mesh, U, 0, tail, cfl, t_stop, scheme, s, closure);
      int64_t launches = chunks * (kGraphSteps / mesh->blocking) + tail;
      if (mesh->blocking == 2 && rest % 2 == 1) {
        // the odd last step as a single step, on the buffers the pairs left
        enqueue_steps(mesh, U, tail, 1, cfl, t_stop, scheme, s, nullptr, tail % 2 == 1);
        ++launches;
      }
      if (scheme == FV_SCHEME_FE && (launches % 2) == 1)
        FV_CUDA(cudaMemcpyAsync(U, mesh->d_work, n * mesh->rec_bytes(), cudaMemcpyDeviceToDevice,
                                s));
      if (mesh->use_lo() && mesh->user_lo) {
        // single steps update the remainder in place; after an odd number of
        // two-step launches it is in the second buffer
        const uint2* last = (mesh->blocking == 2 && tail % 2 == 1) ? mesh->d_lo_stage : mesh->d_lo;
        FV_CUDA(cudaMemcpyAsync(mesh->user_lo, last, n * sizeof(uint2), cudaMemcpyDeviceToDevice,
                                s));
      }
      mesh->last_t_slot = (int)(launches % 2);
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
    if (closure && mesh->f64()) invalid("the learned closure runs on FV_F32 meshes only");
    if (mesh->h.n == 0) return;
    if (!U || !R) invalid("null state or residual");
    if (closure && mesh->wave != FV_WAVE_AVERAGE)
      invalid("the maximum wave speed runs without a closure");
    if (U == R) invalid("R must not alias U");
    cudaStream_t s = as_stream(stream);
    ensure_device(mesh, s);
    fv::StepArgs a = base_args(mesh);
    a.U = U;
    a.out = R;
    // one thread per cell; the tile shape with vertex geometry (same bits)
    const int shape = mesh->vertex_tiles() ? fv::kTileVariant : 0;
    if (shape == fv::kTileVariant) check_tile_smem(mesh, tile_smem(mesh));
    if (closure) {
      ensure_faces(mesh, s);
      FV_CUDA(fv::launch_face_scales(a, mesh->d_faces, mesh->n_faces,
                                     closure_params(mesh, closure), mesh->d_scale, s));
      FV_CUDA(fv::launch_step_scaled(fv::kModeResidual, a, mesh->d_scale, s));
    } else
      FV_CUDA(fv::launch_step(mesh->f64(), fv::kModeResidual, shape, a, s));
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

// ===========================================================================
// Batches of meshes stepped in one launch per step.
// ===========================================================================

struct fv_batch {
  int32_t precision = FV_F32;
  int32_t n_meshes = 0;
  int64_t n = 0;  // padded total cells
  std::vector<int64_t> offsets;      // [n_meshes + 1] start of each mesh's cells
  std::vector<int64_t> mesh_end;     // [n_meshes] one past each mesh's last real cell
  std::vector<int32_t> block_mesh;   // [n / kBlock]
  std::vector<int32_t> first_block;  // [n_meshes + 1]
  std::vector<int32_t> nbr;          // [3n] host staging, global cell ids (-1: padding)
  std::vector<double> nrm;           // [6n]
  std::vector<double> inradius;      // [n]
  std::vector<double> vol;
  std::vector<double> uinf;          // 4 per mesh (conserved)
  bool compensated = true;
  // 0: one thread per cell; 5: TMA-staged tiles; 6: tiles; -1: 6 when its
  // tiles fit in shared memory, else 0 (chosen at the first device call)
  int variant = -1;
  // shared-memory tiles of 1024 cells within each mesh (shape 6)
  bool tiles_ok = false;
  int32_t t1_cap = 0;
  std::vector<int32_t> tile_mesh, tile_cells, mesh_first_tile, tile_info, halo_id;
  std::vector<int64_t> tile_start;
  std::vector<uint32_t> cell_ln;     // [2n]
  // device
  int device = -1;
  bool uploaded = false;
  void* d_nbr = nullptr;
  void* d_geom = nullptr;
  double* d_vol = nullptr;
  void* d_work = nullptr;
  uint2* d_lo = nullptr;
  uint2* d_lo_stage = nullptr;
  void* user_lo = nullptr;  // caller-owned remainder (fv_batch_set_remainder)
  int* d_block_mesh = nullptr;
  int64_t* d_mesh_end = nullptr;
  int* d_first_block = nullptr;
  double* d_uinf = nullptr;
  float* d_uinf_f = nullptr;  // the same rounded to float
  unsigned long long* d_bmin = nullptr;
  double* d_t = nullptr;
  int* d_err = nullptr;
  double* d_partials = nullptr;
  double* d_totals = nullptr;
  int* d_tile_mesh = nullptr;
  int64_t* d_tile_start = nullptr;
  int* d_tile_cells = nullptr;
  int* d_mesh_first_tile = nullptr;
  int* d_tile_info = nullptr;
  int* d_halo_id = nullptr;
  uint2* d_cell_ln = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  const void* g_U = nullptr;
  int32_t g_scheme = -1;
  double g_cfl = 0.0, g_tstop = 0.0;
  bool g_comp = false;
  int g_variant = -1;
  int last_t_slot = 0;
  bool stepped = false;

  bool f64() const { return precision == FV_F64; }
  size_t rec_bytes() const { return f64() ? 32 : 16; }
  bool use_lo() const { return !f64() && compensated; }
  int64_t n_blocks() const { return n / fv::kBlock; }

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
    dev_free(d_block_mesh);
    dev_free(d_mesh_end);
    dev_free(d_first_block);
    dev_free(d_uinf);
    dev_free(d_uinf_f);
    dev_free(d_bmin);
    dev_free(d_t);
    dev_free(d_err);
    dev_free(d_partials);
    dev_free(d_totals);
    dev_free(d_tile_mesh);
    dev_free(d_tile_start);
    dev_free(d_tile_cells);
    dev_free(d_mesh_first_tile);
    dev_free(d_tile_info);
    dev_free(d_halo_id);
    dev_free(d_cell_ln);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
    uploaded = false;
  }
};

namespace {

void batch_ensure_device(fv_batch* b, cudaStream_t s) {
  int dev = 0;
  FV_CUDA(cudaGetDevice(&dev));
  if (b->uploaded) {
    if (dev != b->device) invalid("batch was uploaded to another device");
    return;
  }
  const int64_t n = b->n, nb = b->n_blocks();
  const int M = b->n_meshes;
  FV_CUDA(cudaMalloc(&b->d_nbr, n * (b->f64() ? sizeof(int4) : sizeof(int2))));
  FV_CUDA(cudaMalloc(&b->d_geom, n * 2 * b->rec_bytes()));
  FV_CUDA(cudaMalloc((void**)&b->d_vol, n * sizeof(double)));
  FV_CUDA(cudaMalloc(&b->d_work, n * b->rec_bytes()));
  if (!b->f64()) {
    FV_CUDA(cudaMalloc((void**)&b->d_lo, n * sizeof(uint2)));
    FV_CUDA(cudaMalloc((void**)&b->d_lo_stage, n * sizeof(uint2)));
  }
  FV_CUDA(cudaMalloc((void**)&b->d_block_mesh, nb * sizeof(int)));
  FV_CUDA(cudaMalloc((void**)&b->d_mesh_end, M * sizeof(int64_t)));
  FV_CUDA(cudaMalloc((void**)&b->d_first_block, (M + 1) * sizeof(int)));
  FV_CUDA(cudaMalloc((void**)&b->d_uinf, 4 * M * sizeof(double)));
  FV_CUDA(cudaMalloc((void**)&b->d_uinf_f, 4 * M * sizeof(float)));
  FV_CUDA(cudaMalloc((void**)&b->d_bmin, 3 * M * sizeof(unsigned long long)));
  FV_CUDA(cudaMalloc((void**)&b->d_t, 2 * M * sizeof(double)));
  FV_CUDA(cudaMalloc((void**)&b->d_err, sizeof(int)));
  FV_CUDA(cudaMalloc((void**)&b->d_partials, nb * 4 * sizeof(double)));
  FV_CUDA(cudaMalloc((void**)&b->d_totals, 4 * M * sizeof(double)));
  FV_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  fv::DeviceLayout lay = fv::pack_layout(b->nbr.data(), b->nrm.data(), b->vol.data(),
                                         b->inradius.data(), n, 0, b->f64());
  FV_CUDA(cudaMemcpyAsync(b->d_nbr, lay.nbr.data(), lay.nbr.size(), cudaMemcpyHostToDevice, s));
  FV_CUDA(cudaMemcpyAsync(b->d_geom, lay.geom.data(), lay.geom.size(), cudaMemcpyHostToDevice, s));
  FV_CUDA(cudaMemcpyAsync(b->d_vol, b->vol.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  FV_CUDA(cudaMemcpyAsync(b->d_block_mesh, b->block_mesh.data(), nb * sizeof(int),
                          cudaMemcpyHostToDevice, s));
  FV_CUDA(cudaMemcpyAsync(b->d_mesh_end, b->mesh_end.data(), M * sizeof(int64_t),
                          cudaMemcpyHostToDevice, s));
  FV_CUDA(cudaMemcpyAsync(b->d_first_block, b->first_block.data(), (M + 1) * sizeof(int),
                          cudaMemcpyHostToDevice, s));
  FV_CUDA(cudaMemcpyAsync(b->d_uinf, b->uinf.data(), 4 * M * sizeof(double),
                          cudaMemcpyHostToDevice, s));
  std::vector<float> uinf_f(b->uinf.begin(), b->uinf.end());
  FV_CUDA(cudaMemcpyAsync(b->d_uinf_f, uinf_f.data(), 4 * M * sizeof(float),
                          cudaMemcpyHostToDevice, s));
  FV_CUDA(cudaMemsetAsync(b->d_work, 0, n * b->rec_bytes(), s));
  if (b->tiles_ok) {
    const size_t nt = b->tile_mesh.size(), nh = std::max<size_t>(b->halo_id.size(), 1);
    FV_CUDA(cudaMalloc((void**)&b->d_tile_mesh, nt * sizeof(int)));
    FV_CUDA(cudaMalloc((void**)&b->d_tile_start, nt * sizeof(int64_t)));
    FV_CUDA(cudaMalloc((void**)&b->d_tile_cells, nt * sizeof(int)));
    FV_CUDA(cudaMalloc((void**)&b->d_mesh_first_tile, M * sizeof(int)));
    FV_CUDA(cudaMalloc((void**)&b->d_tile_info, b->tile_info.size() * sizeof(int)));
    FV_CUDA(cudaMalloc((void**)&b->d_halo_id, nh * sizeof(int)));
    FV_CUDA(cudaMalloc((void**)&b->d_cell_ln, n * sizeof(uint2)));
    FV_CUDA(cudaMemcpyAsync(b->d_tile_mesh, b->tile_mesh.data(), nt * sizeof(int),
                            cudaMemcpyHostToDevice, s));
    FV_CUDA(cudaMemcpyAsync(b->d_tile_start, b->tile_start.data(), nt * sizeof(int64_t),
                            cudaMemcpyHostToDevice, s));
    FV_CUDA(cudaMemcpyAsync(b->d_tile_cells, b->tile_cells.data(), nt * sizeof(int),
                            cudaMemcpyHostToDevice, s));
    FV_CUDA(cudaMemcpyAsync(b->d_mesh_first_tile, b->mesh_first_tile.data(), M * sizeof(int),
                            cudaMemcpyHostToDevice, s));
    FV_CUDA(cudaMemcpyAsync(b->d_tile_info, b->tile_info.data(), b->tile_info.size() * sizeof(int),
                            cudaMemcpyHostToDevice, s));
    if (!b->halo_id.empty())
      FV_CUDA(cudaMemcpyAsync(b->d_halo_id, b->halo_id.data(), b->halo_id.size() * sizeof(int),
                              cudaMemcpyHostToDevice, s));
    FV_CUDA(cudaMemcpyAsync(b->d_cell_ln, b->cell_ln.data(), n * sizeof(uint2),
                            cudaMemcpyHostToDevice, s));
  }
  FV_CUDA(cudaStreamSynchronize(s));
  b->device = dev;
  b->uploaded = true;
  if (b->variant < 0) {
    int optin = 0;
    FV_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const bool fits =
        b->tiles_ok && fv::tile_smem_bytes(b->f64(), b->t1_cap) <= (size_t)optin;
    b->variant = fits ? fv::kTileVariant : 0;
  }
}

// Tiles of kBatchTile cells within each mesh of a batch (shape 6), in the
// batch numbering; a mesh whose tiles cannot be built leaves shape 6 off.
void build_batch_tiles(fv_batch* b, fv_mesh* const* meshes) {
  b->cell_ln.assign(2 * (size_t)b->n, 0u);
  b->mesh_first_tile.assign(b->n_meshes, 0);
  try {
    for (int k = 0; k < b->n_meshes; ++k) {
      const fv_mesh* m = meshes[k];
      const int64_t off = b->offsets[k];
      b->mesh_first_tile[k] = (int32_t)b->tile_mesh.size();
      if (m->h.n == 0) continue;
      const fv::PairTiles L = fv::build_pair_tiles(m->h, kBatchTile);
      const int64_t hbase = (int64_t)b->halo_id.size();
      if (hbase + (int64_t)L.halo_id.size() > INT32_MAX) invalid("batch halos too large");
      for (int64_t j = 0; j < L.n_tiles; ++j) {
        b->tile_mesh.push_back(k);
        b->tile_start.push_back(off + j * kBatchTile);
        b->tile_cells.push_back((int32_t)std::min<int64_t>(kBatchTile, m->h.n - j * kBatchTile));
        b->tile_info.push_back((int32_t)(hbase + L.tile_info[2 * j]));
        b->tile_info.push_back(L.tile_info[2 * j + 1]);
      }
      for (int32_t x : L.halo_id) b->halo_id.push_back((int32_t)(x + off));
      std::copy(L.cell_ln.begin(), L.cell_ln.end(), b->cell_ln.begin() + 2 * off);
      b->t1_cap = std::max(b->t1_cap, L.t1_cap);
    }
    b->tile_info.push_back((int32_t)b->halo_id.size());
    b->tile_info.push_back(0);
    b->tiles_ok = true;
  } catch (const fv::Error&) {
    b->tiles_ok = false;
    b->tile_mesh.clear();
    b->tile_start.clear();
    b->tile_cells.clear();
    b->tile_info.clear();
    b->halo_id.clear();
    b->cell_ln.clear();
  }
}

cudaError_t batch_launch(const fv_batch* b, int mode, const fv::BatchArgs& a, cudaStream_t s) {
  if (b->variant == 5) return fv::launch_batch_step_tma(b->f64(), mode, a, s);
  if (b->variant == fv::kTileVariant) return fv::launch_batch_step_tile(b->f64(), mode, a, s);
  return fv::launch_batch_step(b->f64(), mode, a, b->n_blocks(), s);
}

void batch_enqueue_steps(fv_batch* b, void* U, int64_t j0, int64_t count, double cfl,
                         double t_stop, int32_t scheme, cudaStream_t s) {
  for (int64_t j = j0; j < j0 + count; ++j) {
    fv::BatchArgs a{};
    a.s.nbr = b->d_nbr;
    a.s.geom = b->d_geom;
    a.s.n = b->n;
    a.s.cfl = cfl;
    a.s.t_stop = t_stop;
    a.s.err = b->d_err;
    a.s.wait_limit = fv::kDefaultWaitLimit;
    a.s.drain_limit = fv::kDefaultWaitLimit;
    if (b->use_lo()) {
      a.s.lo = b->d_lo;
      a.s.lo_stage = b->d_lo_stage;
    }
    a.block_mesh = b->d_block_mesh;
    a.mesh_end = b->d_mesh_end;
    a.uinf = b->d_uinf;
    a.uinf_f = b->d_uinf_f;
    a.bmin = b->d_bmin;
    a.t = b->d_t;
    a.n_meshes = b->n_meshes;
    a.slot_read = (int)(j % 3);
    a.slot_write = (int)((j + 1) % 3);
    a.slot_reset = (int)((j + 2) % 3);
    a.t_read = (int)(j % 2);
    a.t_write = (int)((j + 1) % 2);
    if (b->variant == fv::kTileVariant) {
      a.s.cell_ln = b->d_cell_ln;
      a.s.tile_info = b->d_tile_info;
      a.s.halo_id = b->d_halo_id;
      a.s.tile = kBatchTile;
      a.s.t1_cap = b->t1_cap;
      a.s.chained = true;
      a.tile_mesh = b->d_tile_mesh;
      a.tile_start = b->d_tile_start;
      a.tile_cells = b->d_tile_cells;
      a.mesh_first_tile = b->d_mesh_first_tile;
      a.n_tiles = (int)b->tile_mesh.size();
    }
    if (scheme == FV_SCHEME_FE) {
      const bool even = (j % 2) == 0;
      a.s.U = even ? U : b->d_work;
      a.s.out = even ? b->d_work : U;
      FV_CUDA(batch_launch(b, fv::kModeFE, a, s));
    } else {
      a.s.U = U;
      a.s.out = b->d_work;
      FV_CUDA(batch_launch(b, fv::kModeRK2a, a, s));
      a.s.U = b->d_work;
      a.s.Ubase = U;
      a.s.out = U;
      FV_CUDA(batch_launch(b, fv::kModeRK2b, a, s));
    }
  }
}

void check_batch(const fv_batch* b) {
  if (!b) invalid("null batch");
}

}  // namespace

extern "C" {

int fv_batch_create(fv_mesh* const* meshes, int32_t n_meshes, fv_batch** out) {
  return guarded([&] {
    if (!out) invalid("null out");
    *out = nullptr;
    if (n_meshes <= 0 || !meshes) invalid("need at least one mesh");
    fv_batch* b = new fv_batch();
    try {
      b->precision = meshes[0] ? meshes[0]->precision : FV_F32;
      b->n_meshes = n_meshes;
      b->offsets.assign(n_meshes + 1, 0);
      for (int k = 0; k < n_meshes; ++k) {
        const fv_mesh* m = meshes[k];
        if (!m) invalid("null mesh in batch");
        if (m->precision != b->precision) invalid("all meshes of a batch need one precision");
        if (m->wave != FV_WAVE_AVERAGE) invalid("batches use the averaged wave speed");
        const int64_t padded = (m->h.n + fv::kBlock - 1) / fv::kBlock * fv::kBlock;
        b->offsets[k + 1] = b->offsets[k] + padded;
      }
      b->n = b->offsets[n_meshes];
      if (b->n == 0) invalid("all meshes are empty");
      if (b->n / fv::kBlock > INT32_MAX || b->n > (int64_t)INT32_MAX)
        invalid("batch too large for 32-bit cell ids");
      const int64_t n = b->n;
      b->nbr.assign(3 * n, -1);
      b->nrm.assign(6 * n, 0.0);
      b->inradius.assign(n, 1.0);  // padding: harmless values, never used
      b->vol.assign(n, 1.0);
      b->uinf.assign(4 * n_meshes, 0.0);
      b->mesh_end.assign(n_meshes, 0);
      b->block_mesh.assign(n / fv::kBlock, 0);
      b->first_block.assign(n_meshes + 1, 0);
      for (int k = 0; k < n_meshes; ++k) {
        const fv_mesh* m = meshes[k];
        const int64_t off = b->offsets[k];
        for (int64_t c = 0; c < m->h.n; ++c) {
          for (int f = 0; f < 3; ++f) {
            const int32_t x = m->h.nbr[3 * c + f];
            b->nbr[3 * (off + c) + f] = x >= 0 ? (int32_t)(x + off) : x;
          }
          for (int f = 0; f < 6; ++f) b->nrm[6 * (off + c) + f] = m->h.nrm[6 * c + f];
          b->inradius[off + c] = m->h.inradius[c];
          b->vol[off + c] = m->h.vol[c];
        }
        b->mesh_end[k] = off + m->h.n;
        m->uinf_conserved(&b->uinf[4 * k]);
        b->first_block[k] = (int32_t)(off / fv::kBlock);
        for (int64_t blk = off / fv::kBlock; blk < b->offsets[k + 1] / fv::kBlock; ++blk)
          b->block_mesh[blk] = k;
      }
      b->first_block[n_meshes] = (int32_t)(n / fv::kBlock);
      build_batch_tiles(b, meshes);
    } catch (...) {
      delete b;
      throw;
    }
    *out = b;
  });
}

int fv_batch_destroy(fv_batch* batch) {
  return guarded([&] {
    if (!batch) return;
    if (batch->uploaded) {
      int cur = 0;
      cudaGetDevice(&cur);
      cudaSetDevice(batch->device);
      cudaDeviceSynchronize();
      batch->free_device();
      cudaSetDevice(cur);
    }
    delete batch;
  });
}

int fv_batch_info(const fv_batch* batch, int64_t* n_cells_padded, int64_t* offsets) {
  return guarded([&] {
    check_batch(batch);
    if (n_cells_padded) *n_cells_padded = batch->n;
    if (offsets)
      std::memcpy(offsets, batch->offsets.data(), batch->offsets.size() * sizeof(int64_t));
  });
}

int fv_batch_set_variant(fv_batch* batch, int32_t variant) {
  return guarded([&] {
    check_batch(batch);
    if (variant != 0 && variant != 5 && variant != fv::kTileVariant)
      invalid("batch kernel shape must be 0, 5 or 6");
    if (variant == fv::kTileVariant) {
      if (!batch->tiles_ok)
        invalid("a mesh of the batch has tiles whose halos exceed 65533 cells; renumber it "
                "with a compact order (Hilbert)");
      int dev = 0, optin = 0;
      FV_CUDA(cudaGetDevice(&dev));
      FV_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      if (fv::tile_smem_bytes(batch->f64(), batch->t1_cap) > (size_t)optin)
        invalid("a tile of the batch with its neighbour ring does not fit in shared memory; "
                "renumber the meshes with a compact order (Hilbert)");
    }
    batch->variant = variant;
    batch->drop_graph();
  });
}

int fv_batch_get_variant(const fv_batch* batch, int32_t* variant) {
  return guarded([&] {
    check_batch(batch);
    if (!variant) invalid("null variant");
    *variant = batch->variant;
  });
}

int fv_batch_set_compensation(fv_batch* batch, int32_t enable) {
  return guarded([&] {
    check_batch(batch);
    if (batch->f64() && enable) invalid("compensated update applies to FV_F32 batches only");
    batch->compensated = enable != 0;
    batch->drop_graph();
  });
}

int fv_batch_set_remainder(fv_batch* batch, void* lo) {
  return guarded([&] {
    check_batch(batch);
    if (lo && batch->f64()) invalid("FV_F64 batches have no remainder");
    batch->user_lo = lo;
  });
}

int fv_batch_step(fv_batch* batch, void* U, int64_t nsteps, double cfl, double t_stop,
                  int32_t scheme, void* stream, double* t_advanced) {
  return guarded([&] {
    check_batch(batch);
    if (nsteps < 0) invalid("nsteps < 0");
    if (scheme != FV_SCHEME_FE && scheme != FV_SCHEME_RK2) invalid("unknown scheme");
    if (!std::isfinite(cfl) || cfl == 0.0) invalid("cfl must be finite and non-zero");
    if (!std::isfinite(t_stop)) invalid("t_stop must be finite");
    if (!U) invalid("null state");
    cudaStream_t s = as_stream(stream);
    batch_ensure_device(batch, s);
    const int M = batch->n_meshes;
    FV_CUDA(fv::launch_batch_init(batch->d_bmin, batch->d_t, M, batch->d_err, s));
    batch->last_t_slot = 0;
    batch->stepped = true;
    if (nsteps > 0) {
      if (batch->use_lo()) {
        if (batch->user_lo)
          FV_CUDA(cudaMemcpyAsync(batch->d_lo, batch->user_lo, batch->n * sizeof(uint2),
                                  cudaMemcpyDeviceToDevice, s));
        else
          FV_CUDA(cudaMemsetAsync(batch->d_lo, 0, batch->n * sizeof(uint2), s));
      }
      if (cfl > 0.0)
        FV_CUDA(fv::launch_batch_bound(batch->f64(), U, batch->d_geom, batch->d_block_mesh,
                                       batch->d_mesh_end, M, batch->n_blocks(), batch->d_bmin,
                                       batch->d_err, s));
      const int64_t chunks = nsteps / kGraphSteps;
      if (chunks > 0) {
        if (!batch->graph || batch->g_U != U || batch->g_scheme != scheme ||
            batch->g_cfl != cfl || batch->g_tstop != t_stop || batch->g_comp != batch->use_lo() ||
            batch->g_variant != batch->variant) {
          batch->drop_graph();
          cudaGraph_t g = nullptr;
          FV_CUDA(cudaStreamBeginCapture(batch->cap_stream, cudaStreamCaptureModeThreadLocal));
          try {
            batch_enqueue_steps(batch, U, 0, kGraphSteps, cfl, t_stop, scheme, batch->cap_stream);
          } catch (...) {
            cudaStreamEndCapture(batch->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
            throw;
          }
          FV_CUDA(cudaStreamEndCapture(batch->cap_stream, &g));
          cudaError_t e = cudaGraphInstantiate(&batch->graph, g, 0);
          cudaGraphDestroy(g);
          FV_CUDA(e);
          batch->g_U = U;
          batch->g_scheme = scheme;
          batch->g_cfl = cfl;
          batch->g_tstop = t_stop;
          batch->g_comp = batch->use_lo();
          batch->g_variant = batch->variant;
        }
        for (int64_t k = 0; k < chunks; ++k) FV_CUDA(cudaGraphLaunch(batch->graph, s));
      }
      const int64_t done = chunks * kGraphSteps;
      batch_enqueue_steps(batch, U, done, nsteps - done, cfl, t_stop, scheme, s);
      if (scheme == FV_SCHEME_FE && (nsteps % 2) == 1)
        FV_CUDA(cudaMemcpyAsync(U, batch->d_work, batch->n * batch->rec_bytes(),
                                cudaMemcpyDeviceToDevice, s));
      if (batch->use_lo() && batch->user_lo)  // updated in place by every step
        FV_CUDA(cudaMemcpyAsync(batch->user_lo, batch->d_lo, batch->n * sizeof(uint2),
                                cudaMemcpyDeviceToDevice, s));
      batch->last_t_slot = (int)(nsteps % 2);
    }
    if (t_advanced) {
      std::vector<double> t(2 * M);
      int err = 0;
      FV_CUDA(cudaMemcpyAsync(t.data(), batch->d_t, 2 * M * sizeof(double),
                              cudaMemcpyDeviceToHost, s));
      FV_CUDA(cudaMemcpyAsync(&err, batch->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
      FV_CUDA(cudaStreamSynchronize(s));
      for (int k = 0; k < M; ++k) t_advanced[k] = t[batch->last_t_slot * M + k];
      if (err & 8)
        throw fv::Error{FV_EINDEX, "a neighbour or halo index was outside its array "
                                   "(bounds-checked build); the state is not valid"};
      if (err & 4)
        throw fv::Error{FV_ESTATE, "a bounded device wait gave up and the copies in flight did "
                                   "not drain either; destroy the batch"};
      if (err & 2)
        throw fv::Error{FV_ETIMEOUT, "a bounded device wait gave up; the state is not valid"};
      if (err) throw fv::Error{FV_ENONFINITE, "a step produced a non-finite state or "
                                              "non-positive density or pressure"};
    }
  });
}

int fv_batch_totals(fv_batch* batch, const void* U, double* out, void* stream) {
  return guarded([&] {
    check_batch(batch);
    if (!U || !out) invalid("null state or out");
    cudaStream_t s = as_stream(stream);
    batch_ensure_device(batch, s);
    FV_CUDA(fv::launch_batch_totals(batch->f64(), U, batch->d_vol, batch->d_block_mesh,
                                    batch->d_mesh_end, batch->d_first_block, batch->n_meshes,
                                    batch->n_blocks(), batch->d_partials, batch->d_totals, s));
    FV_CUDA(cudaMemcpyAsync(out, batch->d_totals, 4 * batch->n_meshes * sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    FV_CUDA(cudaStreamSynchronize(s));
  });
}

}  // extern "C"

// ===========================================================================
// Learned dissipation scale
// ===========================================================================

namespace {

void closure_upload(fv_closure* c, const float* theta, bool on_device, cudaStream_t s) {
  if (theta) {
    FV_CUDA(cudaMemcpyAsync(c->d_theta, theta, fv::kClosureParams * sizeof(float),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  } else {
    FV_CUDA(cudaMemsetAsync(c->d_theta, 0, fv::kClosureParams * sizeof(float), s));
  }
  FV_CUDA(fv::launch_pack_closure(c->d_theta, c->d_w1, c->d_w2, c->d_b, s));
  // b3 is a kernel argument: read it back (a 4-byte copy; synchronises)
  FV_CUDA(cudaMemcpyAsync(&c->b3, c->d_b + 96, sizeof(float), cudaMemcpyDeviceToHost, s));
  FV_CUDA(cudaStreamSynchronize(s));
  static std::atomic<uint64_t> uploads{0};
  c->version = ++uploads;
}

void check_closure(const fv_closure* c) {
  if (!c) invalid("null closure");
}

}  // namespace

extern "C" {

int fv_closure_create(const float* theta, fv_closure** out) {
  return guarded([&] {
    if (!out) invalid("null out");
    *out = nullptr;
    fv_closure* c = new fv_closure();
    try {
      FV_CUDA(cudaGetDevice(&c->device));
      FV_CUDA(cudaMalloc((void**)&c->d_w1, 32 * 4 * sizeof(unsigned)));
      FV_CUDA(cudaMalloc((void**)&c->d_w2, 32 * 16 * sizeof(unsigned)));
      FV_CUDA(cudaMalloc((void**)&c->d_b, 97 * sizeof(float)));
      FV_CUDA(cudaMalloc((void**)&c->d_theta, fv::kClosureParams * sizeof(float)));
      c->grad_blocks = fv::closure_grad_blocks();
      FV_CUDA(cudaMalloc((void**)&c->d_gpart,
                         (size_t)c->grad_blocks * fv::kClosureParams * sizeof(float)));
      FV_CUDA(cudaMalloc((void**)&c->d_lpart, (size_t)c->grad_blocks * sizeof(double)));
      FV_CUDA(cudaMalloc((void**)&c->d_grad, fv::kClosureParams * sizeof(float)));
      FV_CUDA(cudaMalloc((void**)&c->d_loss, sizeof(double)));
      closure_upload(c, theta, false, nullptr);
    } catch (...) {
      cudaFree(c->d_w1);
      cudaFree(c->d_w2);
      cudaFree(c->d_b);
      cudaFree(c->d_theta);
      cudaFree(c->d_gpart);
      cudaFree(c->d_lpart);
      cudaFree(c->d_grad);
      cudaFree(c->d_loss);
      delete c;
      throw;
    }
    *out = c;
  });
}

int fv_closure_destroy(fv_closure* closure) {
  return guarded([&] {
    if (!closure) return;
    cudaDeviceSynchronize();
    cudaFree(closure->d_w1);
    cudaFree(closure->d_w2);
    cudaFree(closure->d_b);
    cudaFree(closure->d_theta);
    cudaFree(closure->d_gpart);
    cudaFree(closure->d_lpart);
    cudaFree(closure->d_grad);
    cudaFree(closure->d_loss);
    delete closure;
  });
}

int fv_closure_set(fv_closure* closure, const float* theta, int32_t theta_on_device,
                   void* stream) {
  return guarded([&] {
    check_closure(closure);
    if (!theta) invalid("null theta");
    closure_upload(closure, theta, theta_on_device != 0, as_stream(stream));
  });
}

int fv_closure_eval(const fv_closure* closure, const float* features, float* scales,
                    int64_t rows, void* stream) {
  return guarded([&] {
    check_closure(closure);
    if (rows < 0) invalid("rows < 0");
    if (rows > 0 && (!features || !scales)) invalid("null features or scales");
    FV_CUDA(fv::launch_closure_eval(features, scales, rows, closure->params(), as_stream(stream)));
  });
}

int fv_closure_scales(fv_mesh* mesh, const void* U, const fv_closure* closure, float* scales,
                      void* stream) {
  return guarded([&] {
    check_mesh(mesh);
    check_closure(closure);
    if (mesh->f64()) invalid("the learned closure runs on FV_F32 meshes only");
    if (mesh->h.n == 0) return;
    if (!U || !scales) invalid("null state or scales");
    cudaStream_t s = as_stream(stream);
    ensure_device(mesh, s);
    ensure_faces(mesh, s);
    fv::StepArgs a = base_args(mesh);
    a.U = U;
    FV_CUDA(fv::launch_face_scales(a, mesh->d_faces, mesh->n_faces, closure_params(mesh, closure),
                                   scales, s));
  });
}

int fv_closure_loss_grad(fv_mesh* mesh, const void* U0, const void* Ut, double dt,
                         const double* weights, fv_closure* closure, double* loss, float* grad,
                         void* stream) {
  return guarded([&] {
    check_mesh(mesh);
    check_closure(closure);
    if (mesh->f64()) invalid("the learned closure runs on FV_F32 meshes only");
    if (!(dt >= 0.0) || !std::isfinite(dt)) invalid("dt must be finite and >= 0");
    if (!weights) invalid("null loss weights");
    for (int q = 0; q < 4; ++q)
      if (!(weights[q] > 0.0) || !std::isfinite(weights[q])) invalid("loss weights must be > 0");
    if (mesh->h.n > 0 && (!U0 || !Ut)) invalid("null state");
    cudaStream_t s = as_stream(stream);
    ensure_device(mesh, s);
    fv::StepArgs a = base_args(mesh);
    a.U = U0;
    FV_CUDA(fv::launch_closure_grad(a, static_cast<const float*>(Ut), dt, weights,
                                    closure->params(), closure->d_gpart, closure->d_lpart,
                                    closure->grad_blocks, closure->d_grad, closure->d_loss, s));
    if (grad)
      FV_CUDA(cudaMemcpyAsync(grad, closure->d_grad, fv::kClosureParams * sizeof(float),
                              cudaMemcpyDeviceToDevice, s));
    if (loss) {
      FV_CUDA(cudaMemcpyAsync(loss, closure->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
      FV_CUDA(cudaStreamSynchronize(s));
    }
  });
}

int fv_restrict_mean(const void* U_fine, int32_t fine_precision, const double* area_fine,
                     const int32_t* fine_of, int64_t n_coarse, int32_t children, void* U_coarse,
                     int32_t coarse_precision, void* stream) {
  return guarded([&] {
    if ((fine_precision != FV_F32 && fine_precision != FV_F64) ||
        (coarse_precision != FV_F32 && coarse_precision != FV_F64))
      invalid("precision must be FV_F32 or FV_F64");
    if (n_coarse < 0 || children < 1 || n_coarse > INT32_MAX / children)
      invalid("bad n_coarse or children");
    if (n_coarse == 0) return;
    if (!U_fine || !area_fine || !fine_of || !U_coarse) invalid("null pointer");
    FV_CUDA(fv::launch_restrict_mean(fine_precision == FV_F64, coarse_precision == FV_F64,
                                     U_fine, area_fine, fine_of, n_coarse, children, U_coarse,
                                     as_stream(stream)));
  });
}

int fv_adam_step(float* theta, const float* grad, float* m, float* v, int64_t n, double lr,
                 double beta1, double beta2, double eps, int64_t step, void* stream) {
  return guarded([&] {
    if (n < 0 || n > INT32_MAX) invalid("bad n");
    if (n > 0 && (!theta || !grad || !m || !v)) invalid("null pointer");
    if (step < 1) invalid("step counts from 1");
    if (!(beta1 >= 0.0 && beta1 < 1.0 && beta2 >= 0.0 && beta2 < 1.0 && eps > 0.0))
      invalid("bad Adam coefficients");
    if (n == 0) return;
    FV_CUDA(fv::launch_adam(theta, grad, m, v, (int)n, lr, beta1, beta2, eps, step,
                            as_stream(stream)));
  });
}

}  // extern "C"
