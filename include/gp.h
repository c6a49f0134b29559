/*
 * gp.h -- C-ABI of the B300 (sm_103a) multilevel CPU/GPU bipartitioner for weighted task DAGs.
 *
 * The operation (Wu, Lohmann, Schroeder-Preikschat, "A Graph-Partition-Based Scheduling Policy for
 * Heterogeneous Architectures"): a task DAG whose vertices carry a CPU and a GPU kernel time and whose
 * edges carry a transfer time, the same in both directions (Sec. III.B), is split into a CPU side and a
 * GPU side (k = 2, Sec. III.B) so that both sides stay within load bounds derived from the workload
 * ratio of Eq. (1)-(2) and the transfer cost of cut edges is small (Sec. IV.C).  The makespan of the
 * resulting mapping is then evaluated exactly.  The multilevel algorithm (the paper delegates it to
 * METIS) is deterministic: results are bit-identical from run to run and to the CPU oracle.
 *
 * Conventions
 *   - vertex ids are int32 (n <= 2^31 - 2); CSR row pointers are int64; times are integer ns.
 *   - part[v] is uint8: 0 = CPU side, 1 = GPU side.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call is stream-ordered and
 *     returns after the results it reports to the host are available.
 *   - "device or host" pointers are classified with cudaPointerGetAttributes; pinned, pageable,
 *     managed and device memory are all accepted there.
 *   - Calls never throw; failures are reported as gp_status.  A gp_graph handle is not thread-safe;
 *     distinct handles may be used from distinct threads.
 *   - All device memory the library allocates comes from the current device's stream-ordered pool.
 */
#ifndef GP_H
#define GP_H
#include <stdint.h>

#if defined(__GNUC__)
#define GP_API __attribute__((visibility("default")))
#else
#define GP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gp_status {
  GP_OK = 0,
  GP_ERR_INVALID = 1,  /* malformed CSR, id out of range, negative cost, bad argument     */
  GP_ERR_NOT_DAG = 2,  /* the graph has a cycle (a self-loop counts as one)               */
  GP_ERR_OOM = 3,      /* a device or host allocation failed                              */
  GP_ERR_CUDA = 4,     /* a CUDA runtime call or kernel launch failed                     */
  GP_ERR_TIMEOUT = 5,  /* a device-side wait exceeded its iteration limit (reserved)       */
  GP_ERR_OVERFLOW = 6  /* a summed cost exceeds 2^61 ns                                   */
} gp_status;

typedef struct gp_graph gp_graph; /* opaque; owns device copies of the DAG */

/* Result of one bipartition. */
typedef struct gp_result {
  int64_t cut;        /* sum of transfer costs of directed edges with ends on different sides   */
  int64_t load_cpu;   /* sum of CPU times of CPU-side vertices                                   */
  int64_t load_gpu;   /* sum of GPU times of GPU-side vertices                                   */
  int64_t bound_cpu;  /* B_C                                                                     */
  int64_t bound_gpu;  /* B_G                                                                     */
  int32_t feasible;   /* load_cpu <= bound_cpu && load_gpu <= bound_gpu                          */
  int32_t levels;     /* number of contractions                                                  */
  int32_t rounds;     /* gain rounds run, summed over levels                                     */
  int32_t coarsest_n; /* vertices of the coarsest graph                                          */
  int64_t alg_bytes;  /* algorithmic bytes moved by the kernels of this call (see DESIGN)        */
  float ms[8];        /* phase times in ms when profiling is on: coarsen, initial, refine, cut   */
} gp_result;

/* Per-level record of the last gp_partition call on a handle (levels 0..levels). */
#define GP_MAX_LEVELS 48
typedef struct gp_trace {
  int32_t levels;
  int32_t gggp_trial;                 /* winning growing trial, -1 when all-GPU was feasible */
  int64_t n[GP_MAX_LEVELS + 1];       /* vertices                                            */
  int64_t a[GP_MAX_LEVELS + 1];       /* adjacency entries                                   */
  int32_t rounds[GP_MAX_LEVELS + 1];  /* gain rounds run at the level                        */
  int64_t moves[GP_MAX_LEVELS + 1];   /* gain-round moves at the level                       */
  int32_t balanced[GP_MAX_LEVELS + 1];/* 1 if a balance round ran                            */
  int64_t bal_moves[GP_MAX_LEVELS + 1];
} gp_trace;

/* ---------------------------------------------------------------------------------------------
 * gp_graph_create -- copy a DAG to the device, validate it, and build what the path needs:
 * the transposed CSR, the undirected weighted graph the cut is measured on (every directed entry
 * u->v of cost w adds w to both W(u,v) and W(v,u): transfer time is direction-free, Sec. III.B),
 * and the topological levels the makespan walks.
 *   n, m       vertex and directed-edge counts (n >= 0, m >= 0)
 *   offsets    int64[n+1] out-CSR row pointers (offsets[0] = 0, offsets[n] = m, non-decreasing)
 *   cols       int32[m]   successor of each edge, in [0, n); parallel entries are allowed
 *   edge_cost  int32[m]   transfer time of each edge (>= 0)
 *   cpu_cost   int32[n]   kernel time on the CPU (>= 0)
 *   gpu_cost   int32[n]   kernel time on the GPU (>= 0)
 *   ptr_kind   0: the five arrays are host memory, 1: device memory of the current device
 *   out        receives the handle; the caller keeps ownership of the inputs (they are copied).
 * Errors: GP_ERR_INVALID, GP_ERR_OVERFLOW, GP_ERR_NOT_DAG (precedence in that order), GP_ERR_OOM,
 * GP_ERR_CUDA, GP_ERR_TIMEOUT.  On error *out is NULL.
 * ------------------------------------------------------------------------------------------- */
GP_API gp_status gp_graph_create(int64_t n, int64_t m, const int64_t* offsets, const int32_t* cols,
                          const int32_t* edge_cost, const int32_t* cpu_cost, const int32_t* gpu_cost,
                          int ptr_kind, void* stream, gp_graph** out);

/* ---------------------------------------------------------------------------------------------
 * gp_graph_create_deferred -- gp_graph_create that returns once the undirected graph is built: the
 * topological levels and the level-ordered in-CSR (which only the makespan, the learned proposal's
 * features and the level export read) are computed on a second stream of the device, on the few
 * SMs a level traversal occupies, while the caller goes on (e.g. with gp_partition, which does not
 * need them).  Arguments as gp_graph_create; the caller must not modify or free the input arrays
 * before the call returns (they are copied).
 * Errors at creation: GP_ERR_INVALID, GP_ERR_OVERFLOW, GP_ERR_NOT_DAG for a self-loop, GP_ERR_OOM,
 * GP_ERR_CUDA.  A cycle through more than one vertex is reported as GP_ERR_NOT_DAG by the first call
 * that waits for the levels: gp_partition (after its split is written), gp_makespan,
 * gp_makespan_noalloc, gp_graph_info (with nlevels), gp_graph_export (with level), the network and
 * learned entry points and the batch entry points; each of them waits for the levels once, and
 * returns the same status for that handle from then on.  gp_graph_destroy waits for them too.
 * ------------------------------------------------------------------------------------------- */
GP_API gp_status gp_graph_create_deferred(int64_t n, int64_t m, const int64_t* offsets, const int32_t* cols,
                                   const int32_t* edge_cost, const int32_t* cpu_cost, const int32_t* gpu_cost,
                                   int ptr_kind, void* stream, gp_graph** out);

GP_API gp_status gp_graph_destroy(gp_graph* g);

/* ---------------------------------------------------------------------------------------------
 * gp_graph_create_batch -- gp_graph_create for `count` DAGs at once: the same checks in the same
 * precedence, the same handle contents, one persistent kernel launch (a CTA builds one DAG at a time,
 * largest first) instead of one call per DAG.  Arrays of `count` entries: n, m, and the five input
 * pointers per DAG (all host memory when ptr_kind = 0, all device memory of the current device when
 * ptr_kind = 1).  out[i] receives DAG i's handle or NULL, status[i] its own status (GP_OK,
 * GP_ERR_INVALID, GP_ERR_OVERFLOW, GP_ERR_NOT_DAG, ...).  The handles are independent: destroy each
 * with gp_graph_destroy (their device memory is one block, freed with the last of them).  DAGs of more
 * than 2^20 vertices are built by gp_graph_create inside the same call.  Returns GP_OK when the call
 * ran (check status[]), GP_ERR_INVALID for malformed arguments, GP_ERR_OOM / GP_ERR_CUDA otherwise.
 * ------------------------------------------------------------------------------------------- */
GP_API gp_status gp_graph_create_batch(int32_t count, const int64_t* n, const int64_t* m,
                                       const int64_t* const* offsets, const int32_t* const* cols,
                                       const int32_t* const* edge_cost, const int32_t* const* cpu_cost,
                                       const int32_t* const* gpu_cost, int ptr_kind, void* stream,
                                       gp_graph** out, gp_status* status);

/* Sizes of a handle: vertices, edges, undirected adjacency entries, topological levels, and the
 * summed CPU / GPU kernel times (SC, SG of Eq. (1)). Any pointer may be NULL. */
GP_API gp_status gp_graph_info(const gp_graph* g, int64_t* n, int64_t* m, int64_t* a0, int32_t* nlevels,
                        int64_t* sum_cpu, int64_t* sum_gpu);

/* Copy out the undirected level-0 graph (compact CSR, rows sorted by neighbour): off int64[n+1],
 * adj int32[a0], W int64[a0]; and the topological level of every vertex, level int32[n]
 * (0 for a vertex without predecessors, else 1 + the largest level of its predecessors).
 * Destinations may be host or device memory; any may be NULL. */
GP_API gp_status gp_graph_export(const gp_graph* g, int64_t* off, int32_t* adj, int64_t* W, int32_t* level,
                          void* stream);

/* ---------------------------------------------------------------------------------------------
 * gp_bounds -- balance bounds from Eq. (1)-(2), exact integers.
 *   r_cpu < 0: Eq. (1) over the summed times: T* = floor(SC*SG/(SC+SG)) (0 when SC+SG = 0), and
 *              B_C = B_G = floor(T* * (1e6 + round(tol*1e6)) / 1e6).
 *   r_cpu in [0, 1]: the CPU takes share r (quantised to 32 fraction bits, Eq. (2) gives the GPU
 *              1 - r): B_C = floor(floor(SC*r) * (1e6+tol_ppm)/1e6), B_G likewise with SG*(1-r).
 *   tol in [0, 1].  Errors: GP_ERR_INVALID for r_cpu > 1 or NaN, tol outside [0, 1], SC or SG < 0.
 * ------------------------------------------------------------------------------------------- */
GP_API gp_status gp_bounds(int64_t sum_cpu, int64_t sum_gpu, double r_cpu, double tol, int64_t* bound_cpu,
                    int64_t* bound_gpu);

/* ---------------------------------------------------------------------------------------------
 * gp_partition -- the multilevel bipartition (coarsening by handshake heavy-edge matching with
 * two-hop pairing, greedy graph growing on the coarsest graph, balance and synchronous gain rounds
 * while uncoarsening).  Balance targets from gp_bounds(SC, SG, r_cpu, tol).
 *   part_out  uint8[n], host or device; receives the split
 *   res       host gp_result, may be NULL
 *   seed      selects the tie-break hash and the growing trials' start vertices
 * An infeasible final split still returns GP_OK with res->feasible = 0.
 * Errors: GP_ERR_INVALID (bad r_cpu/tol, NULL handle or part_out), GP_ERR_OOM, GP_ERR_CUDA.
 * ------------------------------------------------------------------------------------------- */
GP_API gp_status gp_partition(gp_graph* g, double r_cpu, double tol, uint64_t seed, uint8_t* part_out,
                       gp_result* res, void* stream);

/* ---------------------------------------------------------------------------------------------
 * gp_partition_fixed -- gp_partition with fixed vertices.  Sec. III.B roots every initial kernel at
 * an empty kernel whose data sit in host memory; that vertex belongs on the CPU whatever the split.
 *   fixed     int8[n], host or device: 0 pins the vertex to the CPU, 1 to the GPU, -1 leaves it
 *             free; NULL = every vertex free (then exactly gp_partition)
 * Vertices pinned to different sides never merge while coarsening (a coarse vertex is pinned where
 * a member is), the growing starts from the pinned split and moves free vertices only (its all-GPU
 * pre-check becomes: every free vertex on the GPU), and refinement never moves a pinned vertex; so
 * part_out[v] = fixed[v] wherever fixed[v] >= 0.  Pinned loads count toward the bounds: a split
 * they make infeasible returns GP_OK with res->feasible = 0.  The array is read during the call
 * only (the caller keeps it).  Errors: those of gp_partition; GP_ERR_INVALID for a value outside
 * {-1, 0, 1}.
 * ------------------------------------------------------------------------------------------- */
GP_API gp_status gp_partition_fixed(gp_graph* g, const int8_t* fixed, double r_cpu, double tol, uint64_t seed,
                             uint8_t* part_out, gp_result* res, void* stream);

/* Per-level record of the last gp_partition call on g (host struct). */
GP_API gp_status gp_last_trace(const gp_graph* g, gp_trace* trace);

/* ---------------------------------------------------------------------------------------------
 * gp_makespan -- makespan of a mapping with unbounded workers per side:
 *   finish(v) = t_side(v)(v) + max over entries u->v of (finish(u) + [side(u) != side(v)] * w(u,v)),
 *   the max over no entries being 0; makespan = max_v finish(v) (0 when n = 0).
 * Evaluated level by level over the topological levels, in int64.
 *   part        uint8[n] (0/1), host or device
 *   makespan    host int64, receives the result
 *   finish_out  int64[n] host or device, may be NULL; receives finish(v)
 * Errors: GP_ERR_INVALID (NULL arguments or part[v] > 1), GP_ERR_OOM, GP_ERR_CUDA, GP_ERR_TIMEOUT.
 * ------------------------------------------------------------------------------------------- */
GP_API gp_status gp_makespan(const gp_graph* g, const uint8_t* part, int64_t* makespan, int64_t* finish_out,
                      void* stream);

/* ---------------------------------------------------------------------------------------------
 * gp_partition_kway -- k device classes (1 <= k <= 255) by recursive bisection on the 2-way path.
 * The paper names a third processor kind (an FPGA) as future work (Sec. VI) without its costs or a
 * k-class Eq. (1)-(2); this library's reading: every task has one time per class; a group of classes
 * acts as one device whose time for a task folds its classes' times with floor(x*y / (x+y)), left to
 * right; the classes [lo, hi) split into [lo, mid) and [mid, hi), mid = lo + ceil((hi - lo) / 2),
 * by gp_partition on the subgraph induced by the current vertices (group times as its CPU and GPU
 * costs, Eq. (1) bounds from their sums, `tol`, `seed`), recursively; k = 2 is gp_partition.
 *   n, m, offsets, cols, edge_cost   the DAG as in gp_graph_create (ptr_kind: 0 host, 1 device)
 *   costs        int32[k * n], class-major: costs[i * n + v] = v's time on class i (>= 0)
 *   cls_out      uint8[n] (device or host): the class of every vertex
 *   cut          host int64: sum of edge_cost over edges whose ends have different classes
 *   loads        host int64[k]: sum of costs[i * n + v] over the vertices of class i
 *   feasible     host int32 or NULL: 1 if every bisection met its bounds
 *   bisections   host int32 or NULL: bisections run (k - 1 unless a side came out empty)
 * Errors (in this precedence): GP_ERR_INVALID (k, sizes, tol, a negative time, the CSR),
 * GP_ERR_OVERFLOW (a class's or the transfers' sum above 2^61), GP_ERR_NOT_DAG, GP_ERR_OOM,
 * GP_ERR_CUDA, GP_ERR_TIMEOUT.
 * ------------------------------------------------------------------------------------------- */
GP_API gp_status gp_partition_kway(int64_t n, int64_t m, const int64_t* offsets, const int32_t* cols,
                                   const int32_t* edge_cost, int32_t k, const int32_t* costs, int ptr_kind,
                                   double tol, uint64_t seed, uint8_t* cls_out, int64_t* cut, int64_t* loads,
                                   int32_t* feasible, int32_t* bisections, void* stream);

/* ---------------------------------------------------------------------------------------------
 * gp_makespan_workers -- makespan of a mapping on a fixed number of workers per side.  The paper's
 * testbed runs the kernels on 3 CPU worker cores and 1 GPU worker (Sec. IV.A); gp_makespan assumes as
 * many workers as a level needs.  Here every task runs without preemption on one worker of its side
 * for its cost there; its data are there at r(v) = max over in-entries u->v of finish(u) (+ w(u,v)
 * when u is on the other side; every parallel entry counts, transfers do not compete); whenever a
 * worker of a side is idle, the released task of that side with the smallest (r, id) and r <= now
 * starts on it (a list schedule, simulated event by event in time order).  With at least n workers
 * per side the result is gp_makespan's.
 *   part          uint8[n], device or host (0 = CPU, 1 = GPU)
 *   workers_cpu   CPU workers, >= 1; workers_gpu: GPU workers, >= 1; workers_cpu + workers_gpu <= 32
 *   makespan      host int64, receives the largest finish time (0 for an empty graph)
 *   finish_out    int64[n] (device or host) or NULL: every task's finish time
 * The simulation of one graph is sequential (one warp); see gp_batch_makespan_workers for many.
 * Errors: GP_ERR_INVALID (worker counts, part[v] > 1, handle on another device), GP_ERR_OOM,
 * GP_ERR_CUDA, GP_ERR_TIMEOUT (the event loop exceeded its iteration bound).
 * ------------------------------------------------------------------------------------------- */
GP_API gp_status gp_makespan_workers(const gp_graph* g, const uint8_t* part, int32_t workers_cpu,
                                     int32_t workers_gpu, int64_t* makespan, int64_t* finish_out, void* stream);

/* gp_makespan_workers for `count` graphs in one persistent launch (one warp per graph, largest
 * first): parts[i] uint8[n_i] (device or host), makespans int64[count] (host).  Results equal
 * gp_makespan_workers graph by graph. */
GP_API gp_status gp_batch_makespan_workers(int32_t count, gp_graph* const* graphs, const uint8_t* const* parts,
                                           int32_t workers_cpu, int32_t workers_gpu, int64_t* makespans,
                                           void* stream);

/* ---------------------------------------------------------------------------------------------
 * gp_makespan_noalloc -- the same result as gp_makespan, for callers that cannot allocate device
 * memory (the paper has no counterpart: this is a deployment variant).  gp_makespan takes its
 * per-call scratch from the device memory pool.  Hosts that give all device memory to their own
 * allocator at start-up and let no one else allocate (a serving process with its own arenas, a
 * runtime that embeds this library in a fixed memory budget), and latency-critical loops that must
 * not stall on or fail in an allocation, cannot let it.  This variant uses a scratch array compiled
 * into the library (8 MiB + 64 bytes per GPU that loads the library, held until the process exits)
 * and allocates nothing.
 *   g           handle on the current device (GP_ERR_INVALID otherwise)
 *   part        uint8[n] in DEVICE memory (0/1)
 *   makespan    host int64, receives the result
 *   finish_out  int64[n] in DEVICE memory, or NULL
 * The call reads the result back to the host: it synchronises `stream` before it returns.
 * Limits: n <= GP_MAKESPAN_NOALLOC_MAX_N, else GP_ERR_INVALID before any work.  All calls on a GPU
 * share the one scratch array, which keeps the last call's contents: calls whose work overlaps on
 * that GPU (other streams or threads) race; serialise them.  The first call on each device (and the
 * first after that device's context was reset) looks up the array's device address; make that first
 * call before any stream capture begins.
 * Errors: GP_ERR_INVALID (limits, host pointers, part[v] > 1), GP_ERR_CUDA, GP_ERR_TIMEOUT.
 * ------------------------------------------------------------------------------------------- */
#define GP_MAKESPAN_NOALLOC_MAX_N (1 << 20)
GP_API gp_status gp_makespan_noalloc(const gp_graph* g, const uint8_t* part, int64_t* makespan,
                                     int64_t* finish_out, void* stream);

/* ---------------------------------------------------------------------------------------------
 * gp_batch_partition -- gp_partition for `count` graphs in one call.  The paper's scheduler makes
 * its decision offline, one DAG at a time (Sec. IV.D); a scheduler serving many DAGs makes many
 * such decisions, and this entry point makes them together (the paper has no batched form).  Graph i gets exactly what
 * gp_partition(graphs[i], r_cpu[i], tol, seeds[i], parts[i], &res[i], stream) would give it (same
 * split, cut, loads, levels, rounds and coarsest size; ms[] differs).  The graphs run in one
 * persistent kernel launch, replayed from a captured CUDA graph: a CTA takes one graph at a time,
 * largest first, and runs every step of the partition on it.  Graphs with more than 2^23
 * adjacency entries, and graphs whose coarse levels outgrow a CTA's workspace, are partitioned by
 * the single-graph path within the same call.
 *   count       number of graphs (>= 0)
 *   graphs      `count` handles, all on the current device
 *   r_cpu       `count` CPU shares as in gp_partition, or NULL (all -1: Eq. (1) from the sums)
 *   tol         balance tolerance in [0, 1], shared by all graphs
 *   seeds       `count` seeds, or NULL (all 0)
 *   parts       `count` pointers to uint8[n_i] buffers (device or host memory; entries of graphs
 *               with n_i = 0 may be NULL); receive the splits
 *   res         `count` results (host), or NULL; res[i].ms[0] = the persistent kernel's time
 *   makespans   `count` int64 (host) receiving the makespan of each final split (as gp_makespan),
 *               or NULL (the makespan pass is then skipped)
 * The call returns when every output is written (it synchronises `stream`).  Calls on one device
 * are serialised internally.  Errors: GP_ERR_INVALID (arguments, checked before any work),
 * GP_ERR_OOM, GP_ERR_CUDA.
 * ------------------------------------------------------------------------------------------- */
GP_API gp_status gp_batch_partition(int32_t count, gp_graph* const* graphs, const double* r_cpu, double tol,
                                    const uint64_t* seeds, uint8_t* const* parts, gp_result* res,
                                    int64_t* makespans, void* stream);

/* Schedules of the batch kernel (threads per CTA, CTAs per SM, lanes per adjacency row, hash-table
 * size).  A schedule changes only the speed, never a result.
 *   gp_batch_schedule_count: how many there are; gp_batch_schedule_name(i): a short name (NULL
 *   past the last).
 *   gp_batch_set_schedule(i): use schedule i in later calls; -1 restores the default (the
 *   autotuned choice of the device if there is one, else schedule 0).
 *   gp_batch_autotune: runs the batch (arguments as gp_batch_partition; results discarded) once
 *   per schedule after a warm-up run, keeps the fastest as the device's choice, writes its index to
 *   *best and each schedule's kernel time in ms to ms_out[0 .. gp_batch_schedule_count()-1] (if
 *   ms_out != NULL).  Errors as gp_batch_partition. */
GP_API int32_t gp_batch_schedule_count(void);
GP_API const char* gp_batch_schedule_name(int32_t i);
GP_API gp_status gp_batch_set_schedule(int32_t i);
GP_API gp_status gp_batch_autotune(int32_t count, gp_graph* const* graphs, const double* r_cpu, double tol,
                                   const uint64_t* seeds, int32_t* best, float* ms_out, void* stream);

/* Cut of a split: sum of edge costs of directed edges whose ends are on different sides. */
GP_API gp_status gp_cut(const gp_graph* g, const uint8_t* part, int64_t* cut, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Step-level entry points.  They run one step of the path on a caller-supplied undirected level
 * graph held in DEVICE memory, in compact CSR form (off int64[n+1], adj int32[a] sorted within
 * each row, symmetric, no self entries; W int64[a]; vertex weights vC, vG int64[n]).  The caller
 * owns all buffers.  They exist so that each step can be checked on its own.
 * ------------------------------------------------------------------------------------------- */

/* Handshake heavy-edge matching: `rounds` synchronous rounds; each unmatched vertex picks its
 * eligible unmatched neighbour (merged weights within cap_cpu / cap_gpu) with the largest edge
 * under (W desc, h(seed, min, max) desc, min asc, max asc); mutual picks match.  If twohop != 0,
 * the vertices left unmatched are then paired two by two per anchor (best neighbour), walking each
 * anchor's row in neighbour order and skipping pairs over the caps.  mate_out int32[n]: partner or
 * -1. */
GP_API gp_status gp_step_match(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                        const int64_t* vC, const int64_t* vG, int64_t cap_cpu, int64_t cap_gpu,
                        uint64_t seed, int32_t rounds, int32_t twohop, int32_t* mate_out, void* stream);

/* Contraction of a matching: representatives (unmatched, or the smaller of a pair) are numbered in
 * vertex order; cmap_out int32[n]; coarse graph written in compact CSR to coff int64[n+1] (first
 * nc+1 used), cadj int32[a], cW int64[a], cvC / cvG int64[n] (first nc used); *nc_out, *ac_out
 * receive the coarse sizes (host).  Entries within a coarse row are in no particular order (every
 * later step is independent of it). */
GP_API gp_status gp_step_contract(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                           const int64_t* vC, const int64_t* vG, const int32_t* mate, int32_t* cmap_out,
                           int64_t* coff, int32_t* cadj, int64_t* cW, int64_t* cvC, int64_t* cvG,
                           int64_t* nc_out, int64_t* ac_out, void* stream);

/* Greedy graph growing: all-GPU if sum vG <= bound_gpu, else the best of 8 trials; part_out
 * uint8[n] (device), *trial_out (host) = winning trial or -1. */
GP_API gp_status gp_step_gggp(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                       const int64_t* vC, const int64_t* vG, int64_t bound_cpu, int64_t bound_gpu,
                       uint64_t seed, uint8_t* part_out, int32_t* trial_out, void* stream);

/* One growing trial from `start` (0 <= start < n): part_out uint8[n] (device), *cut_out (host). */
GP_API gp_status gp_step_gggp_grow(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                            const int64_t* vC, const int64_t* vG, int64_t bound_cpu, int64_t bound_gpu,
                            int64_t start, uint8_t* part_out, int64_t* cut_out, void* stream);

/* Refinement at one level: a balance round if the split is infeasible, then up to 8 gain rounds
 * (round r moves vertices with positive gain from side r mod 2, in (gain desc, id asc) order, the
 * longest prefix that keeps the destination within its bound), stopping after two consecutive
 * empty rounds.  part (device, uint8[n]) is updated in place.  stats (host int64[6], may be NULL):
 * rounds, balanced, moves, balance moves, load_cpu, load_gpu. */
GP_API gp_status gp_step_refine(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                         const int64_t* vC, const int64_t* vG, int64_t bound_cpu, int64_t bound_gpu,
                         uint8_t* part, int64_t* stats, void* stream);

/* One layer product of the learned proposal's message-passing network (the paper has no network:
 * this is a project addition), on the 5th-generation tensor cores: C[M x N] = A[M x K] . B[K x N]
 * with BF16 inputs and FP32 accumulation, (N, K) in {(64, 192), (192, 64), (64, 64)}.
 *   A  BF16 [M x K] row-major, DEVICE;  B  BF16 [K x N] row-major, DEVICE;  C  FP32 [M x N], DEVICE.
 * Errors: GP_ERR_INVALID (shape, host pointers), GP_ERR_TIMEOUT (a tensor-core wait expired; the
 * kernel released its tensor memory and returned), GP_ERR_OOM, GP_ERR_CUDA. */
GP_API gp_status gp_step_mma_bf16(int64_t M, int32_t N, int32_t K, const void* A, const void* B, float* C,
                                  void* stream);

/* ---------------------------------------------------------------------------------------------
 * Learned proposal (a project addition; the paper's initial split comes from METIS, Sec. III.A).
 * A 3-layer message-passing network (hidden 64) scores every vertex; its logits propose the
 * initial split, and the exact refinement of gp_partition (balance round + gain rounds) runs on
 * level 0 only ("flat mode").  The integer results are exact given the logits.
 *
 * Network: x_v = [log1p(cpu)/16, log1p(gpu)/16, log1p(indeg)/4, log1p(outdeg)/4,
 * level/max(1, levels-1)]; h0 = relu(x W_in + b_in); for l = 1..3,
 * h_l = relu([h | sum_{u->v} e h_u / max(1, indeg) | sum_{v->u} e h_u / max(1, outdeg)] W_l + b_l)
 * with e = log1p(transfer cost)/16 per directed entry; logit = h3 . w_o + b_o.  The layer products
 * run on the tensor cores in BF16 with FP32 accumulation; neighbour sums are order-independent
 * (fixed point), so outputs are deterministic.  Loss: mean binary cross-entropy with the target
 * "the plain method put the vertex on the CPU".  Parameters: GP_MPNN_PARAMS FP32 values in the
 * order W_in(5x64), b_in, W1(192x64), b1, W2, b2, W3, b3, w_o(64), b_o (row-major).
 * ------------------------------------------------------------------------------------------- */
typedef struct gp_model gp_model;
#define GP_MPNN_PARAMS 37505

/* New network on the current device, He-normal weights drawn from splitmix64(seed). */
GP_API gp_status gp_model_create(uint64_t seed, gp_model** out);
GP_API gp_status gp_model_destroy(gp_model* m);
GP_API int64_t gp_model_param_count(void);
/* FP32 parameters to / from host memory (GP_MPNN_PARAMS floats); set resets the optimiser. */
GP_API gp_status gp_model_get_params(const gp_model* m, float* params);
GP_API gp_status gp_model_set_params(gp_model* m, const float* params);
/* Checkpoint: parameters, Adam moments and step: magic "GPMPNN01", uint32 version (2), uint32 parameter
 * count, int64 step, float32 parameters / first / second moments, uint64 FNV-1a checksum of the bytes
 * between the magic and the checksum (all little-endian).  gp_model_load also reads version 1 (no
 * checksum) and rejects a wrong checksum, a truncated or longer file, or a non-finite value with
 * GP_ERR_INVALID. */
GP_API gp_status gp_model_save(const gp_model* m, const char* path);
GP_API gp_status gp_model_load(const char* path, gp_model** out);
/* logits_out: float[n], device or host. */
GP_API gp_status gp_model_forward(const gp_model* m, const gp_graph* g, float* logits_out, void* stream);
/* Gradient of the mean loss on one graph: labels uint8[n] (0 = CPU side, as gp_partition writes it;
 * device or host); grad_out host float[GP_MPNN_PARAMS]; *loss_out the mean loss (may be NULL). */
GP_API gp_status gp_model_grad(gp_model* m, const gp_graph* g, const uint8_t* labels, float* grad_out,
                               double* loss_out, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected) on one graph's gradient. */
GP_API gp_status gp_model_train_step(gp_model* m, const gp_graph* g, const uint8_t* labels, float lr,
                                     double* loss_out, void* stream);
/* The learned path: logits from `logits` (float[n], device or host) when not NULL, else from the
 * network m; vertices ordered by (logit desc, id asc) under the total order of the float bits (a
 * NaN logit is GP_ERR_INVALID); the first k = min(longest prefix whose CPU load fits B_C, shortest
 * prefix after which the GPU load fits B_G) go to the CPU; then the refinement of level 0.  Bounds as
 * gp_partition (Eq. (1)-(2) with tol, or the given ratio).  res: levels = 0, coarsest_n = n,
 * ms[0..2] = network, proposal, refinement + cut (when profiling is on). */
GP_API gp_status gp_partition_learned(gp_graph* g, const gp_model* m, const float* logits, double r_cpu,
                                      double tol, uint8_t* part_out, gp_result* res, void* stream);

/* The learned path as a V-cycle (restricted coarsening): the network's proposal (as above) gives
 * every vertex a side; coarsening matches only vertices proposed to the same side (the sides act as
 * pins for the handshake matching and the two-hop pairing only), so every coarse vertex has one
 * proposed side and the coarsest level takes those sides as its split; every level is then refined
 * on the way back exactly as in gp_partition (projection, balance round, gain rounds, every vertex
 * free).  Arguments as gp_partition_learned, plus `seed` (the matching's tie-break hash, as in
 * gp_partition).  res->ms[4] holds the network and proposal time when profiling is on. */
GP_API gp_status gp_partition_learned_vcycle(gp_graph* g, const gp_model* m, const float* logits, double r_cpu,
                                             double tol, uint64_t seed, uint8_t* part_out, gp_result* res,
                                             void* stream);

/* The learned path for `count` graphs: one network forward over the disjoint union of the graphs,
 * then, per graph, exactly what gp_partition_learned(graphs[i], m, NULL, r_cpu[i], tol, ...) gives
 * it (proposal from the graph's logits, refinement of level 0), run in the persistent batch
 * kernel.  Arguments and outputs as gp_batch_partition (no seeds: the learned path draws nothing).
 * Errors: GP_ERR_INVALID (arguments; a NaN logit; more than 2^31 - 1 entries in the union),
 * GP_ERR_TIMEOUT, GP_ERR_OOM, GP_ERR_CUDA. */
GP_API gp_status gp_batch_partition_learned(int32_t count, gp_graph* const* graphs, const gp_model* m,
                                            const double* r_cpu, double tol, uint8_t* const* parts,
                                            gp_result* res, int64_t* makespans, void* stream);

/* Failure-path self-check of the device waits (no fault involved): one CTA allocates tensor memory
 * as the tensor-core product does, waits on an mbarrier that nothing arrives at with the same bounded
 * wait (limit_ms, 1..2000), gives up, releases the tensor memory and reports it.  Returns
 * GP_ERR_TIMEOUT when the wait gave up as designed (the context stays usable), GP_ERR_INVALID for a
 * limit outside the range. */
GP_API gp_status gp_selftest_wait_timeout(int32_t limit_ms, void* stream);

/* Failure-path self-check of the grid barrier that the wide-level makespan and the large-level
 * refinement use (no fault involved): a cooperative launch of two CTAs in which CTA 1 returns without
 * arriving, so CTA 0's bounded wait (0.5 s) gives up.  Returns GP_ERR_TIMEOUT when it did (the context
 * stays usable), GP_ERR_CUDA if the device has no cooperative launch. */
GP_API gp_status gp_selftest_grid_wait_timeout(void* stream);

/* ---------------------------------------------------------------------------------------------
 * Checked build.  libgp_checked.so is this library compiled with GP_CHECKED: every data-dependent index
 * the kernels gather with (neighbour ids, match partners, coarse ids, successor ids) is tested against
 * its range first; a failed test records its site number in a device word (the first one wins) and the
 * access is skipped, so the results are then meaningless but no access leaves its array.
 * gp_checked_site returns that site (0: none) and clears it when `clear` is nonzero; -1 in the
 * unchecked build.  gp_selftest_checked runs one gather through an out-of-range index behind the test
 * (site 99) and returns GP_OK when the gather was skipped; in the unchecked build it launches nothing
 * and returns GP_ERR_INVALID.
 * ------------------------------------------------------------------------------------------- */
GP_API int32_t gp_checked_site(int32_t clear);
GP_API gp_status gp_selftest_checked(void* stream);

/* ---------------------------------------------------------------------------------------------
 * Instrumentation.
 * gp_launch_count: kernels launched by this library since load (all threads).
 * gp_prof_enable(1): record CUDA events around every launch of each kernel family (on the
 *   launching stream) and accumulate their durations; gp_prof_read returns launches and total ms of
 *   family `kernel` (see gp_kernel_name) and its algorithmic bytes; gp_prof_reset clears them.
 * ------------------------------------------------------------------------------------------- */
GP_API int64_t gp_launch_count(void);
GP_API gp_status gp_prof_enable(int on);
GP_API gp_status gp_prof_reset(void);
GP_API gp_status gp_prof_read(int kernel, int64_t* launches, double* total_ms, int64_t* alg_bytes);
GP_API const char* gp_kernel_name(int kernel); /* NULL past the last family */

GP_API const char* gp_status_string(gp_status s);

#ifdef __cplusplus
}
#endif
#endif
