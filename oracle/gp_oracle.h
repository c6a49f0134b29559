/*
 * gp_oracle.h -- plain, single-threaded CPU oracle of the multilevel CPU/GPU
 * task-DAG bipartitioner and its makespan evaluator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path links, loads or calls
 * this code; only the tests, the package smoke check and the benchmark's CPU
 * baseline leg do.  It shares no source with the CUDA implementation.
 *
 * What it computes (paper: Wu, Lohmann, Schroeder-Preikschat, "A Graph-
 * Partition-Based Scheduling Policy for Heterogeneous Architectures"):
 *   - the weighted task DAG of Sec. III.B (vertex = CPU and GPU kernel time,
 *     edge = transfer time, the same in both directions);
 *   - the workload ratio of Eq. (1)-(2), used as balance targets;
 *   - a 2-way split (k = 2, Sec. III.B) that keeps both sides' loads under
 *     their bounds and minimises the transfer cost of cut edges (Sec. IV.C);
 *   - the makespan of the resulting mapping.
 * The paper hands the split to METIS and does not describe the algorithm; the
 * deterministic multilevel algorithm below (handshake heavy-edge matching,
 * contraction, greedy graph growing, synchronous gain rounds) is this
 * project's reading, written out step by step in the function comments.
 *
 * Conventions: vertex ids int32, CSR row pointers int64, weights int64 above
 * level 0; part[v] = 0 (CPU) or 1 (GPU).  All functions return an OG_* status.
 */
#ifndef GP_ORACLE_H
#define GP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  OG_OK = 0,
  OG_ERR_INVALID = 1,
  OG_ERR_NOT_DAG = 2,
  OG_ERR_OOM = 3,
  OG_ERR_OVERFLOW = 6
};

/* Fixed algorithm constants (they change results). */
#define OG_MATCH_ROUNDS 4     /* handshake rounds per coarsening level        */
#define OG_CAP_DIV 8          /* a coarse vertex may hold at most B/8          */
#define OG_COARSEST 128       /* stop coarsening at <= 128 vertices            */
#define OG_STALL_NUM 95       /* stop when a level keeps > 95/100 of vertices  */
#define OG_STALL_DEN 100
#define OG_MAX_LEVELS 48      /* at most 48 contractions                       */
#define OG_TRIALS 8           /* greedy graph-growing trials                   */
#define OG_REFINE_ROUNDS 8    /* gain rounds per level                         */
#define OG_SUM_LIMIT (((int64_t)1) << 61) /* guard on summed costs             */

typedef struct og_result {
  int64_t cut, load_cpu, load_gpu, bound_cpu, bound_gpu;
  int32_t feasible, levels, rounds, coarsest_n;
} og_result;

/* Per-level record of one partition run (levels 0..levels). */
typedef struct og_trace {
  int32_t levels;              /* number of contractions L                    */
  int32_t gggp_trial;          /* winning trial, -1 when all-GPU was feasible  */
  int64_t n[OG_MAX_LEVELS + 1];
  int64_t a[OG_MAX_LEVELS + 1];          /* adjacency entries               */
  int32_t rounds[OG_MAX_LEVELS + 1];     /* gain rounds run at the level    */
  int64_t moves[OG_MAX_LEVELS + 1];      /* gain-round moves at the level   */
  int32_t balanced[OG_MAX_LEVELS + 1];   /* 1 if a balance round ran        */
  int64_t bal_moves[OG_MAX_LEVELS + 1];
  int64_t cut[OG_MAX_LEVELS + 1];        /* cut after refining the level    */
} og_trace;

typedef struct og_refine_stats {
  int32_t rounds, balanced;
  int64_t moves, bal_moves, load_cpu, load_gpu;
} og_refine_stats;

uint64_t og_mix64(uint64_t z);
uint64_t og_hash(uint64_t seed, uint32_t a, uint32_t b);

int og_validate(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                const int32_t* cpu_cost, const int32_t* gpu_cost);

int og_bounds(int64_t sum_cpu, int64_t sum_gpu, double r_cpu, double tol, int64_t* bound_cpu,
              int64_t* bound_gpu);

int og_symmetrize(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                  int64_t* uoff, int32_t* uadj, int64_t* uW, int64_t* a_out);

int og_match(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
             const int64_t* vC, const int64_t* vG, int64_t cap_cpu, int64_t cap_gpu, uint64_t seed,
             int32_t rounds, int32_t* mate);

int og_match_twohop(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                    const int64_t* vC, const int64_t* vG, int64_t cap_cpu, int64_t cap_gpu,
                    uint64_t seed, int32_t* mate);

int64_t og_count_coarse(int64_t n, const int32_t* mate);

int og_contract(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                const int64_t* vC, const int64_t* vG, const int32_t* mate, int32_t* cmap,
                int64_t* nc_out, int64_t* coff, int32_t* cadj, int64_t* cW, int64_t* cvC,
                int64_t* cvG, int64_t* ac_out);

int og_gggp_grow(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                 const int64_t* vC, const int64_t* vG, int64_t bound_cpu, int64_t bound_gpu,
                 int64_t start, uint8_t* part, int64_t* cut_out);

int og_gggp(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W, const int64_t* vC,
            const int64_t* vG, int64_t bound_cpu, int64_t bound_gpu, uint64_t seed, uint8_t* part,
            int32_t* trial_out);

int og_refine(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
              const int64_t* vC, const int64_t* vG, int64_t bound_cpu, int64_t bound_gpu,
              uint8_t* part, og_refine_stats* st);

int og_partition(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                 const int32_t* cpu_cost, const int32_t* gpu_cost, double r_cpu, double tol,
                 uint64_t seed, uint8_t* part, og_result* res, og_trace* trace);

/* og_partition with fixed vertices (a project addition after Sec. III.B, where every initial kernel
 * depends on an empty kernel whose data sit in host memory): fixed[v] = 0 pins v to the CPU, 1 to the
 * GPU, -1 leaves it free (other values: OG_ERR_INVALID); NULL = all free, i.e. og_partition.  Vertices
 * pinned to different sides never merge, a coarse vertex is pinned where a member is, the growing
 * starts from the pinned split and moves free vertices only, and refinement never moves a pinned
 * vertex, so part[v] = fixed[v] wherever fixed[v] >= 0. */
int og_partition_fixed(int64_t n, int64_t m, const int64_t* off, const int32_t* cols,
                       const int32_t* w, const int32_t* cC, const int32_t* cG, const int8_t* fixed,
                       double r_cpu, double tol, uint64_t seed, uint8_t* part, og_result* res,
                       og_trace* trace);
int og_cut(int64_t n, const int64_t* off, const int32_t* cols, const int32_t* w,
           const uint8_t* part, int64_t* cut);

/* Learned proposal (a project addition; the paper has none): order the vertices by (logit desc,
 * id asc), logits compared as the total order of their IEEE-754 bits (NaN rejected); the first k
 * go to the CPU, k = min(longest prefix with CPU load <= B_C, shortest prefix with GPU load <= B_G). */
int og_propose(int64_t n, const float* logits, const int64_t* vC, const int64_t* vG, int64_t bound_cpu,
               int64_t bound_gpu, uint8_t* part, int64_t* k_out);

/* The learned path: bounds, symmetrised level 0, proposal from the logits, refinement at level 0
 * only (flat mode), cut.  res->levels = 0, res->coarsest_n = n. */
int og_partition_learned(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                         const int32_t* cpu_cost, const int32_t* gpu_cost, const float* logits,
                         double r_cpu, double tol, uint8_t* part, og_result* res);

/* The learned path as a V-cycle (restricted coarsening): the proposal's sides restrict the
 * matching to same-side pairs, the coarsest level takes the proposed sides as its split, and every
 * level is refined on the way back (og_partition's uncoarsening, every vertex free). */
int og_partition_vcycle(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                        const int32_t* cpu_cost, const int32_t* gpu_cost, const float* logits,
                        double r_cpu, double tol, uint64_t seed, uint8_t* part, og_result* res,
                        og_trace* trace);

/* k device classes (1 <= k <= 255) by recursive bisection (Sec. VI's future third processor kind; the
 * project's reading): costs[i * n + v] = v's time on class i; a group of classes acts as one device
 * whose time for v folds its classes' times with floor(x*y / (x+y)); bisect(V', [lo, hi)) splits the
 * subgraph induced by V' with og_partition (cpu_cost = group [lo, mid) with mid = lo + ceil((hi-lo)/2),
 * gpu_cost = group [mid, hi), Eq. (1) bounds from their sums, tol, seed) and recurses on both sides.
 * cls[v] in [0, k); cut over directed entries with different classes; loads[k]; feasible = every
 * bisection feasible; bisections = how many ran. */
int og_partition_kway(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                      int32_t k, const int32_t* costs, double tol, uint64_t seed, uint8_t* cls, int64_t* cut,
                      int64_t* loads, int32_t* feasible, int32_t* bisections);

int og_levels(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, int32_t* level,
              int32_t* nlevels);

int og_makespan(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                const int32_t* cpu_cost, const int32_t* gpu_cost, const uint8_t* part,
                int64_t* finish, int64_t* makespan);

/* Makespan of a mapping on workers_cpu CPU workers and workers_gpu GPU workers (each >= 1; the
 * testbed of Sec. IV.A has 3 and 1): a non-preemptive list schedule simulated in time order.  A task
 * is released when its last predecessor ends and has its data at r(v) (og_makespan's start time);
 * whenever a worker of a side is idle, the released task of that side with the smallest (r, id) and
 * r <= now starts on it.  finish (nullable) receives every task's end time. */
int og_makespan_workers(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                        const int32_t* cpu_cost, const int32_t* gpu_cost, const uint8_t* part,
                        int64_t workers_cpu, int64_t workers_gpu, int64_t* finish, int64_t* makespan);

#ifdef __cplusplus
}
#endif
#endif
