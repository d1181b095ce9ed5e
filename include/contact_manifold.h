/*
 * contact_manifold.h -- C ABI of the GB300 (sm_103a) smooth contact-manifold library.
 *
 * The library evaluates, for many independent body pairs at once, the smoothly
 * differentiable contact manifold of "Smoothly Differentiable and Efficiently
 * Vectorizable Contact Manifold Generation" (arXiv 2602.20304): the map
 * g_{1,2}(pose_1, pose_2) -> {(p_k, d_k, n_k)}_{k=1..K} of Sec. IV-A, built from
 *   - vertex-SDF contacts (Sec. IV-C) of every vertex of each body against the
 *     smooth analytic SDF primitive of the other (Sec. IV-B),
 *   - edge-edge contacts (Sec. IV-D) of every edge pair: the regularised 2x2
 *     box QP solved by the smoothed analytic active set, witness points,
 *     signed distance and normal, and the con/pen/nn/cl activity indicators,
 *   - a SoftSort top-K reduction (Sec. III) of all candidates to K points.
 * Each output point carries a fourth quantity beside (p, d, n): its soft
 * activity weight w.  Rows are laid out (p_x, p_y, p_z, d, n_x, n_y, n_z, w).
 *
 * Conventions shared by every call:
 *   - All pointers named "device" are CUDA device pointers owned by the caller;
 *     the library never frees or retains them past the call (asynchronous
 *     calls read them until the work queued on `stream` completes).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Every compute call is asynchronous on that stream.
 *   - No call aborts the process.  Errors are returned as cm_status and the
 *     message of the last failing call on the calling thread is available from
 *     cm_last_error().  Bad geometry ids found on the device do not fault: the
 *     kernel skips the pair, writes NaN to its output rows and raises a sticky
 *     device flag that cm_check_device_error() reports.
 *   - Floating point is FP32 throughout on the device (the host-side hull
 *     builder, cm_create_hull_geometry, works in double).
 */
#ifndef CONTACT_MANIFOLD_H
#define CONTACT_MANIFOLD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Compile-time limits (validated at cm_create_geometry / on every call). */
#define CM_MAX_K 16        /* contact points per pair */
#define CM_MAX_VERTS 256   /* mesh vertices per geometry */
#define CM_MAX_EDGES 768   /* mesh edges per geometry */
#define CM_MAX_PLANES 512  /* convex-polyhedron planes per geometry */
#define CM_MAX_PRIMS 32    /* superquadrics per SQ_UNION geometry */
#define CM_MAX_SELECT 32   /* soft pre-selected vertices / edges per body */
#define CM_MAX_TRACE 8     /* sphere-tracing steps per witness */
#define CM_MAX_HULL_POINTS 65536 /* input points of cm_create_hull_geometry */

typedef enum {
  CM_OK = 0,
  CM_ERR_INVALID_ARG = 1, /* a size, pointer, id or parameter is out of range */
  CM_ERR_OOM = 2,         /* a device or host allocation failed */
  CM_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
  CM_ERR_ADMISSION = 4,   /* a request does not fit the HBM budget or the device's free memory */
  CM_ERR_TIMEOUT = 5,     /* cm_wait deadline passed before the request finished */
  CM_ERR_NOT_FOUND = 6,   /* unknown geometry id or request ticket */
  CM_ERR_DEVICE = 7       /* a kernel raised the sticky device error flag */
} cm_status;

/* SDF primitive families (Sec. IV-B).  BOX and HULL are convex polyhedra
 * (LSE over planes, Sec. IV-B2); ELLIPSOID is the superquadric with
 * eps1 = eps2 = 1 (Sec. IV-B1); CAPSULE and CYLINDER are smooth readings of the
 * usual primitives (soft-clipped segment distance; LSE of radial and cap
 * distances).  SQ_UNION is a body made of up to CM_MAX_PRIMS general
 * superquadrics joined by the smooth union phi = -LSE_tau(-phi_1, ..., -phi_L)
 * (Sec. IV-B; each phi_l the superquadric SDF of Sec. IV-B1 with exponents
 * eps1, eps2 in [0.1, 1.9]); its normal blends the primitives' grad f with the
 * union's weights softmax(-phi_l / tau).  dims: BOX (hx, hy, hz); CAPSULE
 * (r, h, -); CYLINDER (r, h, -); ELLIPSOID (a, b, c); HULL and SQ_UNION unused. */
enum { CM_BOX = 0, CM_CAPSULE = 1, CM_CYLINDER = 2, CM_ELLIPSOID = 3, CM_HULL = 4, CM_SQ_UNION = 5 };

/* Flags of cm_params.flags: the simplifications of Supplement A, and the
 * non-smoothed witness routines of the paper's Sec. V ablation. */
enum {
  CM_FLAG_NO_EE = 1,      /* vertex-SDF contacts only ("Ours-NE") */
  CM_FLAG_ONE_SIDED = 2,  /* only A's vertices against B's SDF ("Ours-NE-S"); implies NO_EE */
  CM_FLAG_HARD = 4        /* witness-point routines without smoothing ("Ours-NS", Sec. V): hard
                           * clips, argmin and in-box tests; cm_ee_witness_batch and
                           * cm_vf_witness_batch only -- the manifold calls refuse it
                           * (CM_ERR_INVALID_ARG), their operators being the smooth ones */
};

typedef struct cm_context cm_context;

/* A surface in its two representations (Sec. IV-A): mesh and SDF parameters.
 * verts: host, n_verts x 4 floats.  For the analytic primitives each row is a
 *   unit template (u_x, u_y, u_z, s) that maps to a local vertex from the dims
 *   in use: BOX/ELLIPSOID (d0 u_x, d1 u_y, d2 u_z); CYLINDER (r u_x, r u_y, h u_z);
 *   CAPSULE (r u_x, r u_y, r u_z + s h).  For HULL and SQ_UNION the rows are
 *   the vertices.
 * edges: host, n_edges x 2 int32 vertex indices.
 * planes: host.  HULL: n_planes x 4 floats (n_x, n_y, n_z, o) with unit
 *   outward n; the plane value at y is n . y - o.  SQ_UNION: three rows per
 *   superquadric (n_planes = 3 L, 1 <= L <= CM_MAX_PRIMS): (q_w, q_x, q_y, q_z)
 *   its orientation in the body frame (normalised by the library), (t_x, t_y,
 *   t_z, eps1) its centre and first exponent, (a, b, c, eps2) its semi-axes and
 *   second exponent.  NULL / 0 for the other kinds.
 * The library copies everything; the caller may free its arrays on return. */
typedef struct {
  int32_t kind;
  float dims[3];
  int32_t n_verts;
  const float* verts;
  int32_t n_edges;
  const int32_t* edges;
  int32_t n_planes;
  const float* planes;
} cm_geometry_desc;

/* Method parameters.  tau: smoothing of the SDF LSE, soft sign, penetration,
 * nearest-neighbour, clashing and SoftSort operators (used when the per-pair
 * tau pointer is NULL).  w_reg: L2 regulariser of the E-E QP (Sec. IV-D2).
 * eps_clip / eps_min / eps_comp: smoothing of the soft clip, soft argmin and
 * soft comparisons inside the 2x2 box-QP solve.  K: contact points (1..16). */
typedef struct {
  float tau;
  float w_reg;
  float eps_clip;
  float eps_min;
  float eps_comp;
  int32_t K;
  int32_t flags;
  /* Soft top-K pre-selection (Sec. IV-A, the differentiable acceleration
   * structure; Supplement B's safeguard included): when > 0, only the
   * top_verts deepest soft vertices of each body (depth = the other body's SDF)
   * and the top_edges deepest soft edges (depth = mean of the corner depths)
   * generate contacts, each a SoftSort average (temperature tau) of the
   * vertices / edge endpoints; E-E witnesses are then also weighted by the soft
   * indicator of lying inside their own body.  0 keeps all (no selection).
   * At most CM_MAX_SELECT each.  The adjoint differentiates through the
   * selection too (the SoftSort weights through the vertex depths). */
  int32_t top_verts;
  int32_t top_edges;
  /* Sphere tracing of E-E witness points (Supplement, mesh-SDF
   * discrepancies): each witness is moved trace_iters steps x <- x - phi(x) u
   * along the fixed direction u = grad phi / |grad phi| of its own body's SDF at
   * the QP witness; signed distances, normals, penetration and clashing
   * indicators and the output points then use the moved witnesses, while the
   * nearest-neighbour indicators keep the QP witnesses' distances.
   * 0 (default) .. CM_MAX_TRACE; the adjoint differentiates through the
   * unrolled steps and the direction. */
  int32_t trace_iters;
} cm_params;

/* Fills the defaults: tau 1e-2, w_reg 1e-2, eps_* 0.1, K 8, flags 0, no
 * pre-selection, no sphere tracing. */
void cm_default_params(cm_params* p);

/* Creates a context on CUDA device `device`.  hbm_budget_bytes bounds the device
 * memory the context may hold for serving requests (0 = no bound).
 * Returns CM_ERR_CUDA if the device cannot be used.  device = -1 makes a
 * host-only context: geometry can be registered and validated, every call
 * that would touch a device returns CM_ERR_INVALID_ARG. */
cm_status cm_create_context(int device, size_t hbm_budget_bytes, cm_context** out);

/* Waits for the context's work, frees everything it owns.  NULL is ignored. */
void cm_destroy_context(cm_context* ctx);

/* Registers a geometry and returns its id (0, 1, 2, ... in creation order).
 * Validates sizes against the CM_MAX_* limits, finite values, edge indices,
 * dims > 0 for primitives and n_planes >= 4 for hulls.  The packed device copy
 * is uploaded lazily before the next compute call (or by cm_sync_geometry). */
cm_status cm_create_geometry(cm_context* ctx, const cm_geometry_desc* desc, int32_t* geom_id);

/* Uploads pending geometry now (synchronously).  Call before capturing a CUDA
 * graph that launches compute calls, so that the capture contains no copies. */
cm_status cm_sync_geometry(cm_context* ctx);

/* Unregisters geometry `geom_id`: later calls treat a pair that names it like a
 * pair with an unknown id (NaN rows / gradients and the sticky device error
 * flag, see cm_check_device_error).  Ids are never reused and the packed copy
 * keeps the data until the context is destroyed.  Plans made before become
 * invalid.  Destroy only geometry that no call still in flight (including a
 * serving batch) uses.  CM_ERR_INVALID_ARG for an unknown or already destroyed id. */
cm_status cm_destroy_geometry(cm_context* ctx, int32_t geom_id);

/* Number of registered geometries (destroyed ones included: ids are not reused). */
int32_t cm_num_geometries(const cm_context* ctx);

/* Registers the convex hull of a point set as a HULL geometry (Sec. IV-A's two
 * representations of a convex polyhedron: its mesh, and its face planes for the
 * LSE SDF of Sec. IV-B2) and returns its id as cm_create_geometry does.
 * points: host, n_points x 3 doubles, read during the call only;
 *   4 <= n_points <= CM_MAX_HULL_POINTS.
 * The hull is built in double precision and is triangulated: its vertices are the
 * input points on the hull, in input order (a repeated point counts once, at its
 * first index); its edges are the unique edges of the triangles, sorted by
 * (smaller, larger) vertex index; each triangle gives one plane (unit outward
 * normal n, offset n . p), so a flat facet of k triangles gives k equal planes.
 * Points within 1e-9 x the bounding-box diagonal of the hull count as on it.
 * The build is incremental, each point tested against every face of the hull so
 * far: well under a millisecond for a few hundred points, 0.1 s for 65,536
 * points around a small hull, ~30 s for 65,536 points all on a sphere (which
 * then exceed the vertex limit).
 * CM_ERR_INVALID_ARG for non-finite points, fewer than four affinely independent
 * points (all equal, collinear or coplanar), or a hull beyond CM_MAX_VERTS,
 * CM_MAX_EDGES or CM_MAX_PLANES. */
cm_status cm_create_hull_geometry(cm_context* ctx, const double* points, int32_t n_points, int32_t* geom_id);

/* Registers an analytic primitive (Sec. IV-B) with the mesh half of its two
 * representations (Sec. IV-A) generated by the library, `tess` setting its
 * resolution, and returns its id as cm_create_geometry does.  The mesh rows
 * are unit templates (see cm_geometry_desc) scaled by the dims in
 * use, every vertex on the exact surface:
 *   BOX       the 8 corners and 12 edges (tess ignored);
 *   CYLINDER  tess points on each rim (3..128): rim polygons and tess vertical
 *             edges (2 tess vertices, 3 tess edges);
 *   CAPSULE   per cap, rings of tess points (3..63) at latitudes 0 and pi/4 and
 *             a pole: ring polygons, meridian edges ring to ring and ring to
 *             pole, and tess edges joining the equators (4 tess + 2 vertices,
 *             9 tess edges);
 *   ELLIPSOID the icosahedron on the unit sphere subdivided tess times (0..2:
 *             12 / 42 / 162 vertices, 30 / 120 / 480 edges).
 * dims: host, 3 floats as in cm_geometry_desc.  CM_ERR_INVALID_ARG for another
 * kind, tess out of range or dims that cm_create_geometry refuses. */
cm_status cm_create_primitive_geometry(cm_context* ctx, int32_t kind, const float* dims, int32_t tess,
                                       int32_t* geom_id);

/* What cm_get_geometry reports about a registered geometry. */
typedef struct {
  int32_t kind;
  float dims[3];
  int32_t n_verts;
  int32_t n_edges;
  int32_t n_planes; /* HULL: its planes; 0 for every other kind */
} cm_geometry_info;

/* Reads back a registered geometry as the library holds it (both
 * representations of Sec. IV-A: mesh rows and, for hulls, planes).  info (required)
 * gets the kind, registered dims and counts.  Each array that is not NULL gets
 * the data (host memory owned by the caller, sized from the counts of a first
 * call with NULL arrays): verts n_verts x 4 floats (the rows as registered),
 * edges n_edges x 2 int32, planes n_planes x 4 floats (hulls only).
 * CM_ERR_INVALID_ARG for an unknown or destroyed id.  Touches no device. */
cm_status cm_get_geometry(const cm_context* ctx, int32_t geom_id, cm_geometry_info* info, float* verts,
                          int32_t* edges, float* planes);

/* Forward manifold of n_pairs independent pairs (Sec. IV-A's g_{1,2} per pair).
 * pair_geoms: device, n_pairs x 2 int32 geometry ids (A, B).
 * poses: device, n_pairs x 14 floats (qw, qx, qy, qz, tx, ty, tz) of A then B;
 *   the rotation is that of q / |q|.
 * dims: device, n_pairs x 6 floats (dims of A then B) or NULL for each
 *   geometry's registered dims.
 * tau: device, n_pairs floats or NULL for params->tau.
 * out: device, n_pairs x K x 8 floats (p, d, n, w) in world coordinates.
 * n_pairs == 0 is a no-op. */
cm_status cm_contact_manifold_fwd(cm_context* ctx, int32_t n_pairs, const int32_t* pair_geoms,
                                  const float* poses, const float* dims, const float* tau,
                                  const cm_params* params, float* out, void* stream);

/* Adjoint of cm_contact_manifold_fwd (the whole manifold: SDF primitives,
 * QP active set with its soft clips and soft argmin, sign / penetration /
 * nearest-neighbour / clashing indicators, SoftSort).  Same pair arguments as
 * the forward, plus
 * grad_out: device, n_pairs x K x 8, dL/d out in the forward's layout;
 * grad_poses: device, n_pairs x 14, receives dL/d poses (for the raw
 *   quaternion components, i.e. tangent to the unit sphere, and translations);
 * grad_dims: device, n_pairs x 6 or NULL, receives dL/d dims of A then B (the
 *   dims in use; zero for hulls).
 * The forward is recomputed per pair inside the call; nothing is kept between
 * the forward and backward calls. */
cm_status cm_contact_manifold_bwd(cm_context* ctx, int32_t n_pairs, const int32_t* pair_geoms,
                                  const float* poses, const float* dims, const float* tau,
                                  const cm_params* params, const float* grad_out, float* grad_poses,
                                  float* grad_dims, void* stream);

/* Forward records for the adjoint.  cm_contact_manifold_fwd_save is
 * cm_contact_manifold_fwd that also writes, per pair, what the adjoint would
 * otherwise recompute from the whole forward: the K selected SoftSort scores and
 * their candidate ids, the K row normalisers, the K output rows in B's frame and
 * the soft row / column minima of the E-E distance matrix behind the
 * nearest-neighbour indicators (Sec. IV-D3) -- per-pair reductions, never a
 * candidate.  cm_contact_manifold_bwd_saved is cm_contact_manifold_bwd reading
 * them: it skips the forward recompute and evaluates each edge pair's candidates
 * once, in the reverse sweep.  Both calls must see the same pairs, poses, dims,
 * tau and params, with no geometry destroyed in between.
 * saved: device, n_pairs x saved_stride floats, caller-owned; saved_stride (floats
 *   per pair) >= what cm_saved_stride reports for these params and the registered
 *   geometry (it grows with the largest edge count, so registering a geometry
 *   with more edges makes older records too small: the call then returns
 *   CM_ERR_INVALID_ARG).
 * cm_saved_stride: floats per pair for `params` with the geometry registered now. */
cm_status cm_saved_stride(const cm_context* ctx, const cm_params* params, int64_t* floats_per_pair);
cm_status cm_contact_manifold_fwd_save(cm_context* ctx, int32_t n_pairs, const int32_t* pair_geoms,
                                       const float* poses, const float* dims, const float* tau,
                                       const cm_params* params, float* out, float* saved, int64_t saved_stride,
                                       void* stream);
cm_status cm_contact_manifold_bwd_saved(cm_context* ctx, int32_t n_pairs, const int32_t* pair_geoms,
                                        const float* poses, const float* dims, const float* tau,
                                        const cm_params* params, const float* saved, int64_t saved_stride,
                                        const float* grad_out, float* grad_poses, float* grad_dims, void* stream);

/* Candidate dump: every candidate a pair's manifold is reduced from -- the
 * vertex-SDF contacts of Sec. IV-C and both witnesses of every edge pair of
 * Sec. IV-D3 -- as rows (p, d, n, w) in world coordinates, the manifold's own
 * layout, for checking and debugging a manifold candidate by candidate.
 * cm_candidate_offsets (host only, touches no device): offsets_host (n_pairs + 1
 *   int64, caller-owned) receives the first row of each pair (offsets_host[0] = 0,
 *   offsets_host[n_pairs] = total rows) for these params: per pair the vertex
 *   candidates (A's, then B's unless CM_FLAG_ONE_SIDED; with top_verts, that many
 *   selected vertices per body) and, unless CM_FLAG_NO_EE / CM_FLAG_ONE_SIDED,
 *   2 E_A E_B edge candidates (with top_edges, the selected edges).
 *   pair_geoms_host: n_pairs x 2 ids in host memory.  CM_ERR_INVALID_ARG for an
 *   unknown or destroyed id.
 * cm_contact_manifold_fwd_dump: cm_contact_manifold_fwd that also writes pair i's
 *   candidate with id c to row candidate_offsets[i] + c of `candidates` (device,
 *   candidate_rows x 8 floats, caller-owned), ids as the kernels number them: the
 *   vertex candidates first (A's, then B's), then for edge pair (k, l), i.e.
 *   j = k E_B + l, the witness on A's edge at 2 j and the one on B's edge at 2 j + 1.
 *   candidate_offsets: device, n_pairs + 1 int64 from cm_candidate_offsets for the
 *   same pairs and params.  A pair whose range does not match its candidate count,
 *   or passes candidate_rows, writes no rows and sets the context's device error
 *   (cm_check_device_error names it). */
cm_status cm_candidate_offsets(const cm_context* ctx, int32_t n_pairs, const int32_t* pair_geoms_host,
                               const cm_params* params, int64_t* offsets_host);
cm_status cm_contact_manifold_fwd_dump(cm_context* ctx, int32_t n_pairs, const int32_t* pair_geoms,
                                       const float* poses, const float* dims, const float* tau,
                                       const cm_params* params, float* out, float* candidates,
                                       int64_t candidate_rows, const int64_t* candidate_offsets, void* stream);

/* Batching layer (not part of the paper's method).
 *
 * cm_autotune times a few launch shapes (threads per CTA, CTAs per SM, with or
 * without the size-ordered work list) of the forward -- and of the adjoint
 * when grad_out is given -- on this batch, and keeps the fastest for later
 * calls with the same direction, batch-size bucket (power of two), largest
 * edge count (bucket of 32) and flags.  It runs the kernels several times,
 * overwrites out / grad_poses / grad_dims, and synchronises `stream`.
 * cm_get_launch_shape reports the shape a call would use. */
cm_status cm_autotune(cm_context* ctx, int32_t n_pairs, const int32_t* pair_geoms, const float* poses,
                      const float* dims, const float* tau, const cm_params* params, float* out,
                      const float* grad_out, float* grad_poses, float* grad_dims, void* stream);
cm_status cm_get_launch_shape(const cm_context* ctx, int32_t n_pairs, int32_t backward, int32_t flags,
                              int32_t* block, int32_t* ctas_per_sm, int32_t* ordered);

/* A plan is the steady-state step of one fixed batch -- work ordering, forward
 * and (when grad_out != NULL) adjoint -- captured once into a CUDA graph with
 * its own scratch, then replayed by cm_plan_launch with a single graph launch.
 * The plan keeps the device pointers it was made with: the caller updates the
 * contents of poses / dims / tau / grad_out in place between launches and
 * reads out / grad_poses / grad_dims after the launch completes on `stream`.
 * Registering new geometry invalidates plans (cm_plan_launch then returns
 * CM_ERR_INVALID_ARG).  Plans of one context may run concurrently on
 * different streams; each owns its scratch.  cm_plan_create synchronises. */
typedef struct cm_plan cm_plan;
cm_status cm_plan_create(cm_context* ctx, int32_t n_pairs, const int32_t* pair_geoms, const float* poses,
                         const float* dims, const float* tau, const cm_params* params, float* out,
                         const float* grad_out, float* grad_poses, float* grad_dims, cm_plan** plan);
cm_status cm_plan_launch(cm_plan* plan, void* stream);
void cm_plan_destroy(cm_plan* plan);

/* Serving (not part of the paper's method): a scheduler thread per context
 * continuously batches requests from many clients.  Requests are admitted in
 * arrival order as the context's HBM budget (cm_create_context), the device's
 * free memory (cudaMemGetInfo plus what the stream-ordered pool holds unused,
 * less a 256 MiB reserve) and the batch pair limit allow; a request that does
 * not fit the free memory while none of the server's batches is running fails
 * with CM_ERR_ADMISSION (from cm_wait / cm_poll).  Each admitted group becomes
 * one batch (forward over all
 * its pairs, adjoint over the pairs of forward+backward requests) issued on
 * one of n_streams streams, so batches formed while others run overlap on the
 * GPU.  Geometry stays resident; pair data is copied in and results copied out
 * per request.  All requests of one server agree on whether they give dims
 * and tau.  Host buffers of a request (pinned memory recommended) must stay
 * valid until the request is done. */
typedef struct {
  int32_t n_pairs;        /* 1..max_batch_pairs */
  int32_t with_backward;  /* 0: forward only; 1: forward + adjoint */
  const int32_t* pair_geoms; /* host, n x 2 */
  const float* poses;        /* host, n x 14 */
  const float* dims;         /* host, n x 6, or NULL (registered dims) */
  const float* tau;          /* host, n, or NULL (the server's params.tau) */
  const float* grad_out;     /* host, n x K x 8 (with_backward) */
  float* out;                /* host, n x K x 8, written on completion */
  float* grad_poses;         /* host, n x 14 (with_backward) */
  float* grad_dims;          /* host, n x 6 or NULL */
} cm_request_desc;

/* Starts the serving loop of `ctx` with fixed method params.  Returns
 * CM_ERR_ADMISSION if the budget cannot hold one batch's scratch. */
cm_status cm_server_start(cm_context* ctx, const cm_params* params, int32_t max_batch_pairs, int32_t n_streams);
/* Queues a request; CM_ERR_ADMISSION if it cannot fit the budget even alone. */
cm_status cm_submit(cm_context* ctx, const cm_request_desc* req, uint64_t* ticket);
/* Non-blocking: *done = 1 once the request's results are in its host buffers. */
cm_status cm_poll(cm_context* ctx, uint64_t ticket, int32_t* done);
/* Blocks up to timeout_ms; CM_ERR_TIMEOUT if the request is still running. */
cm_status cm_wait(cm_context* ctx, uint64_t ticket, int32_t timeout_ms);
/* Submission-to-completion time of a finished request, in seconds. */
cm_status cm_request_latency(cm_context* ctx, uint64_t ticket, double* seconds);
/* Forgets a finished request (its ticket becomes unknown). */
cm_status cm_release(cm_context* ctx, uint64_t ticket);
/* Pairs and batches completed so far and device bytes currently admitted. */
cm_status cm_server_stats(cm_context* ctx, uint64_t* pairs_done, uint64_t* batches_done, uint64_t* bytes_in_use);
/* Drains queued and running requests, then stops the loop. */
cm_status cm_server_stop(cm_context* ctx);

/* Same manifold and arguments as cm_contact_manifold_fwd, but the call
 * allocates no memory (no cudaMalloc, no library allocation).  The paper has no
 * counterpart.  It is for callers that cannot allocate while they run the
 * manifold: a host application that hands out every device allocation from its
 * own pool (so its accounting and limit stay exact), or a real-time loop that
 * was promised a fixed memory footprint and cannot absorb the blocking and
 * synchronisation of cudaMalloc / cudaFree.  Its E-E distance scratch is one
 * fixed 64 MiB device array (16 Mi floats) in the library, present on every GPU
 * that loads the library until the process exits.
 *   - It keeps one scratch float per edge pair (the distance) and solves each
 *     witness QP a second time in pass 2, where the regular forward keeps four
 *     floats per edge pair and reads the QP back: same results, more arithmetic.
 *   - Limit: the largest registered geometry may have at most
 *     floor(sqrt(16 Mi / number_of_SMs)) edges (332 on a 152-SM GB300), so that
 *     a max_e^2 slice fits per SM; otherwise CM_ERR_INVALID_ARG with a message
 *     stating the limit.  Parameters are validated as cm_contact_manifold_fwd
 *     validates them (the same K and flag checks).
 *   - Geometry must already be uploaded (cm_sync_geometry); a pending upload is
 *     an error here instead of an allocation.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and sets the kernel's shared-memory limit; make that
 *     first call before any stream capture.
 *   - Every call, from any context, shares the one array per device and it keeps
 *     the last call's contents: calls whose kernels overlap on the GPU (other
 *     streams, other threads) race on it and must be serialised by the caller.
 *     Every entry a call reads it has written first, so nothing needs clearing. */
cm_status cm_contact_manifold_fwd_noalloc(cm_context* ctx, int32_t n_pairs, const int32_t* pair_geoms,
                                          const float* poses, const float* dims, const float* tau,
                                          const cm_params* params, float* out, void* stream);

/* Reads (and clears) the sticky device error flag; synchronises the context's
 * default work.  Returns CM_ERR_DEVICE with a message naming the first bad pair
 * when a kernel met an invalid geometry id. */
cm_status cm_check_device_error(cm_context* ctx);

/* Witness-point routines on their own, for independent queries (the paper's
 * witness-point throughput setting, Sec. V, Fig. 6).  Device buffers, 16-byte
 * aligned; they run on the current device and need no context.  With
 * CM_FLAG_HARD in params->flags both run the same analytic active set without
 * smoothing (the paper's Ours-NS): the exact box-QP minimiser (con = 1 when the
 * unconstrained one is inside the box, else 0) and the exact closest point of the
 * triangle (inside = 1 or 0); ties between sides go to the first in the order
 * a1 = 1, a1 = 0, a2 = 1, a2 = 0 (E-E) and t0t1, t1t2, t0t2 (V-F).
 * cm_ee_witness_batch: queries n x 12 floats (a0, a1 of edge 1; b0, b1 of edge 2);
 *   the regularised 2x2 box QP with the smoothed analytic active set (Sec. IV-D2)
 *   using params->w_reg and eps_*; out n x 8 floats (e1*, e2*, con, |e1* - e2*|).
 * cm_vf_witness_batch: queries n x 12 floats (v, t0, t1, t2); the smoothed closest
 *   point of the triangle to v (Sec. IV-D1: plane projection blended with the
 *   soft-argmin of the soft-clipped edge projections by the soft barycentric
 *   inside test); out n x 4 floats (witness, inside indicator). */
cm_status cm_ee_witness_batch(int32_t n, const float* queries, const cm_params* params, float* out, void* stream);
cm_status cm_vf_witness_batch(int32_t n, const float* queries, const cm_params* params, float* out, void* stream);

/* Measures the device's FP32 FMA throughput (flop/s, 2 per FMA) and MUFU ex2
 * throughput (op/s) with two short synthetic kernels on `device`; used as the
 * denominators of the arithmetic roofline.  Not part of the paper's method. */
cm_status cm_measure_pipe_peaks(int device, double* fma_flops, double* mufu_ops);

/* Message of the last failing call on this thread ("" if none). */
const char* cm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CONTACT_MANIFOLD_H */
