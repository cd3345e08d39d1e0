/*
 * fv.h -- C ABI of the GB300 library for the explicit cell-centred
 * finite-volume step of the 2D Euler equations on triangles with the
 * Lax-Friedrichs flux (Nagy et al., "Accelerating unstructured finite volume
 * computations on field-programmable gate arrays", Sec. 6 and Sec. 7).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an int status (FV_OK = 0 or an FV_E* code).  On
 *   failure fv_last_error() returns a message for the calling thread; nothing
 *   else is changed unless the function says so.
 * - Handles (fv_mesh, fv_batch, fv_closure) are opaque and owned by the
 *   library until their *_destroy call.
 * - State arrays are caller-owned device memory: n_cells records of four
 *   values (rho, rho*u, rho*v, E) in the mesh precision (float for FV_F32,
 *   double for FV_F64), record c at offset 4*c -- the conserved vector U of
 *   Sec. 6.1.  The library never frees caller memory.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Work is queued on it; only functions that return host values
 *   (totals, time, status) synchronise it.
 * - A mesh is built on the host; its device arrays are created on first
 *   device use (or by fv_mesh_upload) on the current CUDA device, so the
 *   host-side functions work on a machine without a GPU.  Device use of one
 *   handle from several host threads at once is not supported.
 * - Cell numbering: after fv_renumber, cell i of the mesh is the cell that
 *   was number perm[i] before the call; states must be permuted alike.
 */
#ifndef FV_H_
#define FV_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define FV_OK 0
#define FV_EINVAL 1     /* bad argument or malformed mesh */
#define FV_ENOMEM 2     /* host or device allocation failed */
#define FV_ECUDA 3      /* a CUDA runtime call failed (message has the CUDA error) */
#define FV_ENONFINITE 4 /* a step produced a non-finite state, rho <= 0 or p <= 0 */
#define FV_ETIMEOUT 5   /* a bounded device wait gave up */
#define FV_ESTATE 6     /* a bounded device wait gave up and the kernel's own bulk copies
                           still in flight did not complete within the drain limit either:
                           they may still write the device memory of the mesh or batch.
                           Destroy the handle (and do not reuse its state buffers). */
#define FV_EINDEX 7     /* bounds-checked builds only (see fv_index_checks): a kernel met a
                           neighbour, halo or node index outside the array it indexes, skipped
                           that access and flagged it; the state is not valid. */

/* ---- precision of a mesh's state and geometry ------------------------------ */
#define FV_F32 0
#define FV_F64 1

/* ---- boundary tags of fv_mesh_create's bnd_edges (reading of Sec. 7, where
 * ghost cells carry the inflow, outflow and wall conditions) ---------------- */
#define FV_BC_NONE 0     /* no default: an unmatched edge is an error */
#define FV_BC_WALL 1     /* slip wall: ghost mirrors the normal momentum */
#define FV_BC_FARFIELD 2 /* far field: ghost is the free stream of fv_set_freestream */
#define FV_BC_EXTRAP 3   /* extrapolation: ghost copies the interior state */

/* ---- cell orders of fv_renumber (Sec. 4: renumbering for data locality) --- */
#define FV_ORDER_IDENTITY 0
#define FV_ORDER_SHUFFLE 1 /* uniform random permutation from the seed */
#define FV_ORDER_RCM 2     /* reverse Cuthill-McKee from a pseudo-peripheral cell */
#define FV_ORDER_HILBERT 3 /* Hilbert curve through the cell centroids */
#define FV_ORDER_AM1 4     /* Amoeba1, the paper's serial-bandwidth heuristic (Sec. 4.2) */

/* ---- time schemes of fv_step ----------------------------------------------- */
#define FV_SCHEME_FE 0  /* forward Euler, Eq. 6 and the update equation of Sec. 6.2.2 */
#define FV_SCHEME_RK2 1 /* two-stage Heun (SSP-RK2) with the same dt; not in the paper */

/* Where the step kernel takes face normals and areas from (fv_mesh_set_geometry) */
#define FV_GEOM_STORED 0 /* per-cell records computed on the host (Sec. 7: precomputed) */
#define FV_GEOM_VERTEX 1 /* formed from node coordinates on a fixed-point grid (Sec. 7) */

/* Tensor-core engine of the learned closure's MLP (fv_mesh_set_closure_engine) */
#define FV_CLOSURE_MMA_SYNC 0 /* warp-level mma.sync m16n8k16, registers */
#define FV_CLOSURE_TCGEN05 1  /* tcgen05.mma, 128-row tiles, accumulator in TMEM */

/* Wave speed in the Lax-Friedrichs dissipation (fv_mesh_set_wave_speed) */
#define FV_WAVE_AVERAGE 0 /* |average normal velocity| + average sound speed (Sec. 6.2.2) */
#define FV_WAVE_MAX 1     /* max over both sides of |normal velocity| + sound speed */

typedef struct fv_mesh fv_mesh;
typedef struct fv_batch fv_batch;
typedef struct fv_closure fv_closure;

/* Message of the last failed call on this thread ("" if none).  The pointer
 * stays valid until the next failing call on the same thread. */
const char* fv_last_error(void);

/* ABI version of this header: 1. */
int32_t fv_abi_version(void);

/* 1 if this library is the bounds-checked build (compiled with FV_DEBUG),
 * else 0.  In that build every kernel tests each index it reads through a
 * table -- global neighbour ids against the cell count, 16-bit tile-local ids
 * against the entries its tile staged in shared memory, halo ids, node ids --
 * and on an index outside its array skips the access and sets an error bit
 * that fv_step and fv_mesh_status report as FV_EINDEX (fv_batch_step for
 * batches).  It stands in for a memory checker on machines where none can
 * run; results are bitwise those of the normal build. */
int32_t fv_index_checks(void);

/* ===========================================================================
 * Mesh (Sec. 6.2.1 geometry; Sec. 7: each cell has three neighbours, ghost
 * cells at boundaries; face sizes and normals are precomputed).
 * ======================================================================== */

/* Builds a mesh on the host.
 *   xy[2*n_nodes]      node coordinates (x, y), host, read only.
 *   tri[3*n_tri]       node ids per triangle, host; clockwise triangles are
 *                      reoriented; face k of a triangle is the edge from its
 *                      vertex k to vertex k+1 (mod 3) after reorientation.
 *   node_canon         nullable, [n_nodes]: node -> node it is identified with
 *                      (periodic domains).  Edges are matched on these ids.
 *                      Each face has one normal (Sec. 7 precomputes face sizes
 *                      and normals), taken from the coordinates of the cell
 *                      whose (smaller, larger) node-id pair of that edge is the
 *                      smaller one; the other cell uses its negation.
 *   bnd_edges[3*n_bnd] nullable: (node a, node b, FV_BC_* tag) for edges that
 *                      border no other cell.
 *   default_bc         FV_BC_* tag for unmatched edges not in bnd_edges.
 *   precision          FV_F32 or FV_F64.
 * Errors: FV_EINVAL for a zero-area or non-finite triangle, an edge shared by
 * more than two cells, an edge collapsed by node_canon, an out-of-range node
 * id, or an unmatched edge without a tag.  The free stream defaults to
 * rho = 1, u = v = 0, p = 1.  *out receives the handle. */
int fv_mesh_create(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
                   const int32_t* node_canon, const int32_t* bnd_edges, int64_t n_bnd,
                   int32_t default_bc, int32_t precision, fv_mesh** out);

/* Frees the host and device arrays of the mesh (waits for its device work). */
int fv_mesh_destroy(fv_mesh* mesh);

/* Number of cells and precision of a mesh. */
int fv_mesh_info(const fv_mesh* mesh, int64_t* n_cells, int32_t* precision);

/* Free-stream primitive state (rho, u, v, p) used by far-field ghosts.
 * rho and p must be positive and finite. */
int fv_set_freestream(fv_mesh* mesh, double rho, double u, double v, double p);

/* Renumbers the cells (Sec. 4) and remaps the neighbour table; each cell keeps
 * its local face order.  perm_out (nullable, host, [n_cells]) receives the
 * permutation new -> old relative to the numbering before this call.  seed is
 * used by FV_ORDER_SHUFFLE only.  Device arrays are refreshed on next use. */
int fv_renumber(fv_mesh* mesh, int32_t order, uint64_t seed, int32_t* perm_out);

/* Locality diagnostics of the current numbering on the cell graph (Sec. 4.1):
 * the bandwidth B_f(G) = max |f(u) - f(v)| over neighbouring cells, and the
 * serial bandwidth S_BW = max_i E(i) - S(i) (nullable outputs). */
int fv_mesh_diagnostics(const fv_mesh* mesh, int64_t* bandwidth, int64_t* serial_bandwidth);

/* Host copies of the built geometry in the current numbering (nullable):
 *   nbr[3*n]     neighbour across each face, or -FV_BC_* for a ghost face
 *   normals[6*n] outward face normal times face length, (x, y) per face
 *   area[n]      triangle area V_T */
int fv_mesh_export(const fv_mesh* mesh, int32_t* nbr, double* normals, double* area);

/* FV_F32 meshes: chooses how fv_step adds each increment to the float state.
 * enable = 1 (the default): compensated -- the part of every update that the
 * float state cannot represent is kept in a per-cell bfloat16 remainder
 * (8 bytes per cell, library-owned and zeroed at the start of every fv_step
 * call, unless the caller supplies it with fv_mesh_set_remainder) and added
 * back on the next step, so long runs do not stall when increments fall below
 * half a float ulp of the state.  enable = 0: plain float update.
 * Not part of the paper; FV_EINVAL for FV_F64 meshes with enable = 1. */
int fv_mesh_set_compensation(fv_mesh* mesh, int32_t enable);

/* Caller-owned remainder of the compensated FP32 update, so that a run split
 * over several fv_step calls, or saved to a checkpoint and resumed later,
 * gives the same bits as one call.  Not part of the paper.
 *   lo  device memory of n_cells records of 8 bytes: four bfloat16 values per
 *       cell, the remainders of rho, rho*u, rho*v, E in U's order, in the
 *       mesh's current cell numbering; or NULL (the default): the library's
 *       own remainder, zeroed at the start of every fv_step call.
 * With lo set, each fv_step call starts from the remainder in lo and leaves
 * the remainder of its final state there (two device-to-device copies of
 * 8 bytes per cell per call).  The library never clears lo: zero it whenever
 * a new state is put into U -- a zero remainder is the state of a fresh
 * start, and a call with a zeroed lo gives the bits of a call without one.
 * Saving U and lo and loading both resumes a run bit for bit.  lo must stay
 * valid while it is set; after fv_renumber permute it as U.  It is not read
 * or written while compensation is off.  FV_EINVAL for a non-NULL lo on an
 * FV_F64 mesh. */
int fv_mesh_set_remainder(fv_mesh* mesh, void* lo);

/* Shape of the step kernel: 0 one thread per cell; 1 (default) a persistent
 * grid of resident blocks that walks the cells and prefetches the next
 * cell's records; 2 the same limited to 64 registers per thread; 3 and 4 one
 * thread per cell limited to 40 and 32 registers; 5 a persistent grid whose
 * cell records are staged in shared memory by bulk (TMA) copies; 6 tiles of
 * consecutive cells (the tile size of fv_mesh_set_blocking, default 1024)
 * whose states and primitive variables, with those of the tile's neighbour
 * ring, sit in shared memory, so each primitive is formed once per cell (the
 * tile arrays are built on the host at the next device call; FV_EINVAL from
 * fv_step if a tile with its ring does not fit in shared memory); 7 the tile
 * shape evaluating each face once: the cell that owns a face writes its flux
 * to its own slot and the exact negation to the slot of the cell across (the
 * face fluxes are antisymmetric bit for bit), then every cell adds its three
 * slots -- half the face arithmetic, for three flux records per tile cell of
 * shared memory (forward Euler and RK2; the residual runs as shape 0; not
 * with FV_GEOM_VERTEX).  All give bitwise identical results; only speed
 * differs.  FV_EINVAL outside 0..7. */
int fv_mesh_set_variant(fv_mesh* mesh, int32_t variant);

/* Times every step-kernel shape on this mesh (a few steps each on a device
 * copy of U with a negligible fixed dt; U itself is not changed), keeps the
 * fastest for later fv_step calls and reports it in *best (nullable);
 * us_per_step (nullable, host, [8]) receives the measured microseconds per
 * step of each shape (infinity for a tiled shape when its tiles do not fit).
 * Shapes 6 and 7 are timed with tiles of 256, 384, 512, 768, 1024 and 2048
 * cells (and sizes that fill whole waves) and reported at their best; when one wins, its
 * tile size is kept (the tile size is shared with fv_mesh_set_blocking).  Allocates and frees one state-sized device buffer
 * and synchronises the stream. */
int fv_mesh_autotune(fv_mesh* mesh, const void* U, int32_t scheme, void* stream, int32_t* best,
                     double* us_per_step);

/* Polls of a device-side wait before it gives up (shape 5 waits for its bulk
 * copies on mbarriers).  A wait that gives up makes the kernel stop, drain its
 * own copies in flight (with the default limit) and set an error bit, and
 * fv_step / fv_mesh_status return FV_ETIMEOUT; the state is then not valid.
 * If the drain gives up as well they return FV_ESTATE.
 * Default 2^24.  A limit of 0 forces the timeout path (for tests). */
int fv_mesh_set_wait_limit(fv_mesh* mesh, uint32_t polls);

/* Wave speed of the dissipation term of Eq. 5.  FV_WAVE_AVERAGE (default) is
 * the paper's: the absolute interface-average normal velocity plus the
 * average sound speed.  FV_WAVE_MAX takes the larger one-sided
 * |u_n| + c of the two cells (the Rusanov form).  The paper's averages can
 * fall below the one-sided speeds in strong expansions, where the first-order
 * update then loses positivity (the corner of the Mach 3 forward-facing step
 * on fine meshes); the maximum keeps it positive under the same CFL bound.
 * With FV_WAVE_MAX the step runs shape 0, 1, 6 or 7 (shapes 2-5 run as 1);
 * fv_step returns FV_EINVAL with a closure or two steps per launch, and
 * fv_batch_create with such a mesh.  FV_EINVAL for an unknown mode. */
int fv_mesh_set_wave_speed(fv_mesh* mesh, int32_t mode);

/* Normals from vertex coordinates: the alternative the paper weighs against
 * stored normals for its FPGA design (Sec. 7), trading bytes per cell for
 * arithmetic.  FV_F32 meshes; the tile shape (6) of the step kernel.
 *   form  FV_GEOM_STORED (default): every step kernel reads each cell's
 *         precomputed normals and 1/V (32 bytes per cell in FP32).
 *         FV_GEOM_VERTEX: the tile kernel stages the grid coordinates of its
 *         tile's nodes in shared memory (8 bytes per node, about half a node
 *         per cell) and forms each cell's three normals from them, reading
 *         4 bytes of node ids and 4 of 1/V per cell instead of 32 of
 *         geometry.
 * The first FV_GEOM_VERTEX call snaps every node of the mesh to a grid of
 * spacing s = 2^e, the finest with the mesh's extent E within 2^31 - 16
 * steps (so a node moves by at most s, s <= E / (2^31 - 16)); a periodic node
 * copy keeps the offset of its canonical node in whole steps.  Normals and
 * areas of the mesh are then those of the snapped nodes for every shape,
 * every later call and any batch made from the mesh: normals are exact
 * integer edge vectors times 2^e, which the kernel converts to FP32 with one
 * rounding -- bitwise the stored FP32 normals -- and 2V is an exact 64-bit
 * cross product; so all shapes still give bitwise the same states.  The
 * snapping stays when
 * the form goes back to FV_GEOM_STORED.  fv_mesh_nodes returns the snapped
 * coordinates.  Selecting FV_GEOM_VERTEX also selects shape 6; fv_mesh_autotune
 * then times shape 6 at each tile size only.
 * FV_EINVAL: an FV_F64 mesh, an unknown form, or a mesh that the grid cannot
 * hold (extent outside 2^-62 .. 2^62 times 2^31, coordinates too far from the
 * origin for exact FP64 grid points, a triangle that collapses on the grid,
 * or a face whose two sides are not exact opposites after snapping, e.g. an
 * inconsistent periodic identification); the mesh is unchanged then. */
int fv_mesh_set_geometry(fv_mesh* mesh, int32_t form);

/* Host diagnostics of the vertex geometry (after FV_GEOM_VERTEX): the nodes
 * that the tile kernel stages for tile `tile` (cells [tile*tile_cells,
 * (tile+1)*tile_cells) of the current numbering), in the order of the
 * tile-local node ids.  All outputs nullable, host.
 *   grid_xy     [2*capacity] their grid coordinates (x, y): a node sits at
 *               centre + grid_xy * 2^e (fv_mesh_nodes gives e).
 *   n_nodes     number of nodes of the tile.
 *   cell_local  [3 * cells of the tile] each cell's three tile-local node
 *               ids, counter-clockwise (face k runs from node k to k+1).
 * FV_EINVAL without vertex geometry, for a bad tile index or size, or a
 * capacity below n_nodes. */
int fv_mesh_tile_nodes(const fv_mesh* mesh, int32_t tile_cells, int64_t tile, int32_t* grid_xy,
                       int64_t capacity, int64_t* n_nodes, uint16_t* cell_local);

/* Node coordinates of the mesh as its geometry uses them: those given to
 * fv_mesh_create, or after FV_GEOM_VERTEX their grid points (nodes that no
 * triangle uses keep their coordinates).  All outputs nullable, host.
 *   n_nodes        number of nodes.
 *   xy             [2*n_nodes] (x, y) per node.
 *   grid_exponent  e of the grid spacing 2^e, or INT32_MIN if not snapped. */
int fv_mesh_nodes(const fv_mesh* mesh, int64_t* n_nodes, double* xy, int32_t* grid_exponent);

/* Launch chaining of the step kernels (default 1 = on): each step kernel of
 * fv_step is launched with programmatic dependent launch, so the next step's
 * launch is prepared while the current step runs and its blocks wait in
 * hardware for the current step to complete before reading anything; this
 * hides most of the launch gap between steps.  Results are identical either
 * way; 0 launches each step in plain stream order (for comparison). */
int fv_mesh_set_launch_chaining(fv_mesh* mesh, int32_t enable);

/* Two time steps per launch: temporal blocking, the GPU form of the paper's
 * chaining of processors, where the output of one update feeds the next
 * without another pass through memory (Sec. 7).  FV_F32 meshes, forward
 * Euler, no closure.
 *   steps_per_launch  1 (default: one fused kernel per step) or 2.
 *   tile_cells        cells per tile: 0 (= 1024), 512, 768, 1024 or 2048
 *                     with 2; with 1, 0 or any size from 32 to 2048 for the
 *                     one-step tile shape (6), which fv_mesh_autotune also
 *                     sets (it times sizes that fill whole waves of resident
 *                     blocks besides the standard four).
 *   staged            0: one block per tile, records loaded through the
 *                     caches; 1: persistent blocks whose tile records arrive
 *                     by bulk copies into double-buffered shared memory
 *                     (tiles of 512 or 1024 cells; its waits are bounded as
 *                     set by fv_mesh_set_wait_limit, FV_ETIMEOUT if one gives
 *                     up; the state pointer must be 16-byte aligned).
 * With 2, each launch stages a tile of consecutive cells plus its two rings
 * of neighbours in shared memory and advances the tile by two steps.  The
 * cell arithmetic is that of the one-step kernel, so with a fixed dt
 * (cfl < 0 in fv_step) the result is bitwise that of single steps.  With
 * cfl > 0 both steps of a pair use the CFL bound of the state at the start
 * of the pair (dt evaluated every second step).  An odd last step runs as a
 * single step.  Halos must fit in shared memory: renumber with a compact
 * order first (FV_ORDER_HILBERT); fv_step returns FV_EINVAL otherwise.
 * fv_step then also returns FV_EINVAL for RK2 or a closure.  Returns
 * FV_EINVAL for FV_F64 meshes with 2, a tile size outside those above, or
 * tiles of 2048 cells with staged = 1. */
int fv_mesh_set_blocking(fv_mesh* mesh, int32_t steps_per_launch, int32_t tile_cells,
                         int32_t staged);

/* The step-kernel shape (0-6) and the tile size in cells of the tiled shapes
 * that the mesh runs now (set by fv_mesh_set_variant, fv_mesh_set_blocking,
 * fv_mesh_set_geometry or fv_mesh_autotune).  Outputs nullable, host. */
int fv_mesh_get_tiling(const fv_mesh* mesh, int32_t* variant, int32_t* tile_cells);

/* Host diagnostics of the two-step tiles: the halos of tile `tile` (cells
 * [tile*tile_cells, (tile+1)*tile_cells) of the current numbering).
 * halo_ids (nullable, host, `capacity` entries) receives the first halo (the
 * cells outside the tile adjacent to it) then the second (cells outside tile
 * and first halo adjacent to the first halo), each in ascending id;
 * n_first / n_second their sizes.  FV_EINVAL for a bad tile index, a
 * capacity below n_first + n_second, or a tile with halos above 65533 cells. */
int fv_mesh_tile_halo(const fv_mesh* mesh, int32_t tile_cells, int64_t tile, int32_t* halo_ids,
                      int64_t capacity, int64_t* n_first, int64_t* n_second);

/* ===========================================================================
 * Partitioning for several processes (host only).  Part p of nparts owns the
 * contiguous range [p*n/nparts, (p+1)*n/nparts) of the current numbering
 * (renumber first: RCM or Hilbert ranges are compact).  Its local numbering is
 * the owned cells in global order followed by its halo: every other cell that
 * an owned cell has as a neighbour, in ascending global id.  Stepping a part
 * needs the halo states from their owners after every stage and the minimum
 * of the CFL bound over all parts (the paper's design is one FPGA; several
 * FPGAs are its future work, Sec. 8).
 * ======================================================================== */

/* Sizes of part `part`: owned cells and halo cells. */
int fv_partition_sizes(const fv_mesh* mesh, int32_t nparts, int32_t part, int64_t* n_owned,
                       int64_t* n_halo);

/* Host arrays of part `part` (all nullable):
 *   global_ids[n_owned + n_halo]  local -> global cell id
 *   halo_owner[n_halo]            part that owns each halo cell
 *   nbr[3 * n_owned]              neighbours in local ids (ghost codes < 0)
 *   normals[6 * n_owned], area[n_owned]  geometry of the owned cells */
int fv_partition_local(const fv_mesh* mesh, int32_t nparts, int32_t part, int64_t* global_ids,
                       int32_t* halo_owner, int32_t* nbr, double* normals, double* area);

/* Creates or refreshes the device arrays now, on `stream` (otherwise the
 * first device call does it).  Allocates device memory. */
int fv_mesh_upload(fv_mesh* mesh, void* stream);

/* Test support of the bounds-checked build (FV_EINVAL in the normal build):
 * overwrites one entry of the mesh's device neighbour tables so that a test
 * can check that the kernels catch an index outside its array.
 *   table 0: the global neighbour id of face `slot` (0..2) of `cell`;
 *   table 1: its 16-bit tile-local id (tiles must have been built by a step
 *            of a tiled shape; value 0..0xFFFF).
 * Synchronises the stream.  The host mesh is unchanged; fv_renumber or a new
 * tile size rebuilds the device tables from it. */
int fv_mesh_debug_set_index(fv_mesh* mesh, int32_t table, int64_t cell, int32_t slot,
                            int32_t value, void* stream);

/* ===========================================================================
 * Time stepping (Eq. 4 semi-discrete form, Eq. 5 flux, Eq. 6 forward Euler).
 * ======================================================================== */

/* Advances U in place by up to nsteps steps.
 *   U        device, [4*n_cells] in the mesh precision.
 *   cfl      > 0: each step uses dt = cfl * min_T 2 V_T / (P_T (|v_T| + c_T))
 *            on the state at the start of the step (P_T the perimeter; the
 *            paper does not define dt); < 0: fixed dt = -cfl.
 *   t_stop   > 0: the time advanced in this call stops at t_stop (the last dt
 *            is clamped, later steps advance nothing); <= 0: no limit.
 *   scheme   FV_SCHEME_FE or FV_SCHEME_RK2.
 *   closure  nullable: learned dissipation scale per face (fv_closure_*);
 *            FV_F32 meshes only.  With shape 7 (fv_mesh_set_variant; tiles
 *            of up to 1024 cells) the learned step runs as one kernel per
 *            stage on the tiles, each face's features, scale and flux formed
 *            once; otherwise as a pass over the mesh's faces for the scales
 *            and a step that reads them.  Both give the same bits.
 *   t_advanced nullable host pointer: if given, the call synchronises the
 *            stream, stores the time advanced, and returns FV_ENONFINITE if a
 *            step produced a bad state.  If NULL nothing is synchronised; use
 *            fv_mesh_status to collect the outcome later.
 * The step loop runs as captured CUDA graphs of one fused kernel per step;
 * the first call with a new (U, scheme, cfl, t_stop, closure) captures them. */
int fv_step(fv_mesh* mesh, void* U, int64_t nsteps, double cfl, double t_stop, int32_t scheme,
            const fv_closure* closure, void* stream, double* t_advanced);

/* Waits for the stream and reports the last fv_step: time advanced (nullable)
 * and FV_ENONFINITE if a bad state was seen. */
int fv_mesh_status(fv_mesh* mesh, void* stream, double* t_advanced);

/* R = dU/dt = -(1/V_T) sum_f F_f |n_f| (Eq. 4) for the state U; both device
 * arrays of [4*n_cells] in the mesh precision; R must not alias U. */
int fv_residual(fv_mesh* mesh, const void* U, void* R, const fv_closure* closure, void* stream);

/* dt of the next step for state U (see fv_step's cfl), written to the host
 * double *dt; synchronises the stream. */
int fv_compute_dt(fv_mesh* mesh, const void* U, double cfl, void* stream, double* dt);

/* Conserved totals sum_T V_T U_T (mass, x and y momentum, energy; Eq. 1a-1c)
 * accumulated in FP64 in a fixed order (bitwise reproducible for a given
 * numbering), written to host out[4]; synchronises the stream. */
int fv_conserved_totals(fv_mesh* mesh, const void* U, double* out, void* stream);

/* ===========================================================================
 * Learned dissipation scale (not in the paper).  Per face, an MLP
 * 8 -> 32 -> 32 -> 1 with ReLU maps eight features of the two states that do
 * not change when the cells are swapped (|jump of rho| / mean rho,
 * |jump of u_n| / c-bar, |jump of u_t| / c-bar, |jump of p| / mean p,
 * |mean u_n| / c-bar, |jump of u_n / c|, min c / c-bar, max c / c-bar) to
 * s = 0.2 + 1.3 sigmoid(z), which multiplies the dissipation term of Eq. 5.
 * Hidden-layer weights are bfloat16 (features and hidden activations are
 * rounded to bfloat16 as tensor-core operands), accumulation is FP32.  Runs
 * on FV_F32 meshes (FV_EINVAL otherwise).
 * ======================================================================== */

/* theta: host FP32, 1377 values in the order W1[32][8] (row = hidden unit),
 * b1[32], W2[32][32], b2[32], w3[32], b3; NULL = all zero.  Allocates device
 * memory on the current device. */
int fv_closure_create(const float* theta, fv_closure** out);

/* Frees the closure's device memory (waits for the device); NULL is a no-op.
 * Step graphs that meshes captured with it are never replayed again: every
 * closure carries a process-unique parameter stamp, so another closure, even
 * at the same address, makes the mesh recapture. */
int fv_closure_destroy(fv_closure* closure);

/* New parameters (same order); theta is host memory, or device memory when
 * theta_on_device != 0.  Synchronises the stream.  A mesh whose captured
 * step graph used the closure recaptures it on its next fv_step (the output
 * bias b3 is a kernel argument of the captured launches). */
int fv_closure_set(fv_closure* closure, const float* theta, int32_t theta_on_device,
                   void* stream);

/* The MLP alone: features device FP32 [rows][8] -> scales device FP32 [rows]. */
int fv_closure_eval(const fv_closure* closure, const float* features, float* scales,
                    int64_t rows, void* stream);

/* The scale of every face for state U: device FP32 [3 * n_cells], face k of
 * cell c at 3c + k. */
int fv_closure_scales(fv_mesh* mesh, const void* U, const fv_closure* closure, float* scales,
                      void* stream);

/* Tensor-core engine of the MLP in this mesh's learned steps (fv_step,
 * fv_residual, fv_closure_scales; both the two-pass form and the one kernel
 * on shape 7's tiles).  FV_CLOSURE_MMA_SYNC (default): a warp evaluates 16
 * rows per mma.sync, accumulators in registers.  FV_CLOSURE_TCGEN05: 128
 * threads evaluate 128 rows per tcgen05.mma from shared-memory operands into
 * tensor memory (32 columns per 128 rows), each thread reading its row back;
 * waits on the MMAs are bounded by fv_mesh_set_wait_limit (FV_ETIMEOUT /
 * FV_ESTATE as for shape 5).  Both engines give the same bits.  The training
 * kernels (fv_closure_loss_grad, fv_closure_eval) use mma.sync.  FV_EINVAL for
 * an unknown engine. */
int fv_mesh_set_closure_engine(fv_mesh* mesh, int32_t engine);

/* Training signal of the closure: one forward-Euler step with fixed dt from
 * U0 (device FP32 [4n]) with the closure, compared with the target Ut:
 *   L = sum_T V_T sum_q ((U0 + dt R(U0) - Ut)_q / weights[q])^2
 * weights: host double[4] (> 0).  loss: host double (nullable; if given, the
 * stream is synchronised).  grad: device FP32 [1377] dL/dtheta in the order of
 * fv_closure_create (nullable), differentiated through the bfloat16 roundings
 * as if they were the identity.  Deterministic (fixed reduction order). */
int fv_closure_loss_grad(fv_mesh* mesh, const void* U0, const void* Ut, double dt,
                         const double* weights, fv_closure* closure, double* loss, float* grad,
                         void* stream);

/* Restriction of a fine state to a coarse mesh (training data of the
 * closure): coarse cell c gets the area-weighted mean of its `children` fine
 * cells, sum_j V_j U_j / sum_j V_j over j = fine_of[c*children + 0 ..
 * children-1], accumulated in FP64 in that order.
 *   U_fine    device, fine states in fine_precision (FV_F32 / FV_F64).
 *   area_fine device double [fine cells]: the fine cells' areas.
 *   fine_of   device int32 [n_coarse * children]: fine cell ids (in the
 *             numbering of U_fine) of each coarse cell (in the numbering of
 *             U_coarse), e.g. the 16 children of two midpoint refinements.
 *   U_coarse  device, [4*n_coarse] in coarse_precision, written.
 * Ids are not checked on the device: every id must index U_fine and
 * area_fine.  FV_EINVAL for an unknown precision, children < 1 or a null
 * pointer.  Nothing is synchronised. */
int fv_restrict_mean(const void* U_fine, int32_t fine_precision, const double* area_fine,
                     const int32_t* fine_of, int64_t n_coarse, int32_t children, void* U_coarse,
                     int32_t coarse_precision, void* stream);

/* One Adam update (Kingma and Ba) of n device FP32 parameters with moments m,
 * v (device, caller-owned, start at zero); step counts from 1. */
int fv_adam_step(float* theta, const float* grad, float* m, float* v, int64_t n, double lr,
                 double beta1, double beta2, double eps, int64_t step, void* stream);

/* ===========================================================================
 * Batches: many independent meshes of uneven size advanced by one launch per
 * step (not in the paper).  The meshes' cells are concatenated, each mesh's
 * range padded to a multiple of 256 cells, so every thread block works on one
 * mesh; each mesh keeps its own dt (its own CFL minimum), time and free
 * stream, and advances bit for bit as it would alone in the same precision.
 * ======================================================================== */

/* Copies the current geometry, numbering and free streams of the meshes
 * (all of one precision; the meshes may be destroyed afterwards).
 * FV_EINVAL for no meshes, mixed precisions or more than 2^31 cells. */
int fv_batch_create(fv_mesh* const* meshes, int32_t n_meshes, fv_batch** out);

/* Frees the batch's host and device arrays (waits for its device work); NULL
 * is a no-op.  The meshes it was made from are not touched. */
int fv_batch_destroy(fv_batch* batch);

/* Padded total number of cells, and offsets[n_meshes + 1] (nullable): mesh k
 * owns records offsets[k] .. offsets[k] + n_cells(k) - 1 of the batch state;
 * the records up to offsets[k + 1] are padding, ignored and unspecified. */
int fv_batch_info(const fv_batch* batch, int64_t* n_cells_padded, int64_t* offsets);

/* Kernel shape of a batch: 5 TMA-staged 256-cell tiles, one per block of the
 * batch (see fv_mesh_set_variant); 0 one thread per cell; 6 tiles of 1024
 * cells within each mesh with their neighbour ring and primitives in shared
 * memory (needs compactly numbered meshes: FV_EINVAL if a tile's ring does
 * not fit).  Default: 6 when its tiles fit, else 0 (decided at the first
 * device call).  All give bitwise identical results. */
int fv_batch_set_variant(fv_batch* batch, int32_t variant);

/* The batch's kernel shape in *variant: 0, 5 or 6, or -1 while the default
 * is still to be decided at the first device call. */
int fv_batch_get_variant(const fv_batch* batch, int32_t* variant);

/* Compensated float update for FV_F32 batches (see fv_mesh_set_compensation). */
int fv_batch_set_compensation(fv_batch* batch, int32_t enable);

/* Caller-owned remainder of a batch's compensated update, as
 * fv_mesh_set_remainder: lo holds n_cells_padded records of 8 bytes (device),
 * in the batch's record order; NULL returns to the library's own remainder,
 * zeroed at the start of every fv_batch_step call.  FV_EINVAL for a non-NULL
 * lo on an FV_F64 batch. */
int fv_batch_set_remainder(fv_batch* batch, void* lo);

/* fv_step for every mesh of the batch: U is device memory of n_cells_padded
 * records in the batch precision; cfl, t_stop and scheme apply to every mesh,
 * dt is each mesh's own.  t_advanced (nullable, host, [n_meshes]): if given the
 * call synchronises, stores each mesh's time advanced and returns
 * FV_ENONFINITE if any state went bad.  Device arrays are created on first use. */
int fv_batch_step(fv_batch* batch, void* U, int64_t nsteps, double cfl, double t_stop,
                  int32_t scheme, void* stream, double* t_advanced);

/* Per-mesh conserved totals, host out[4 * n_meshes], FP64, fixed order;
 * synchronises the stream. */
int fv_batch_totals(fv_batch* batch, const void* U, double* out, void* stream);

/* ===========================================================================
 * Allocation-free variant.  The paper has no counterpart: this is a service
 * entry point for callers that cannot allocate device memory.
 * ======================================================================== */

/* Conserved totals sum_T V_T U_T, like fv_conserved_totals, for callers that
 * must not allocate device memory -- for example code that runs inside a
 * framework whose caching allocator owns the whole device memory budget, or a
 * latency-critical loop where cudaMalloc's implicit device synchronisation
 * would stall other streams.  It calls no cudaMalloc, cudaFree or allocating
 * library routine and needs no fv_mesh.
 *   U        device, [4*n_cells] states in `precision` (FV_F32 or FV_F64),
 *            16-byte aligned for FV_F32 and 32-byte aligned for FV_F64.
 *   area     device, [n_cells] cell areas V_T (e.g. fv_mesh_export's area,
 *            copied to the device by the caller), same cell order as U,
 *            8-byte aligned.
 *   out      device, double[4], written by the call (caller-owned), 8-byte
 *            aligned.
 *   stream   cudaStream_t as void*; nothing is synchronised.
 * Scratch: per-tile partial sums live in a fixed array inside the library's
 * device code (4096 tiles of 4096 cells, 128 KiB per GPU, held by every GPU
 * that loads the library until the process exits).  Hence n_cells may be at
 * most 16,777,216; larger sizes, a null or misaligned pointer and an unknown
 * precision return FV_EINVAL before any device work.
 * Every call looks up that array's device address (cudaGetSymbolAddress) for
 * the current device, so a device reset between calls is harmless; the first
 * call on a device also loads the library's device code there, so make that
 * first call before any stream capture.  All calls share the one array:
 * calls that overlap on the GPU (different streams, no ordering) race and
 * give wrong sums.  Every partial a call reads is written earlier in the same
 * call, so leftovers of a previous call do not matter.  Results agree with
 * fv_conserved_totals to rounding (the summation order differs). */
int fv_conserved_totals_noalloc(const void* U, const double* area, int64_t n_cells,
                                int32_t precision, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FV_H_ */
