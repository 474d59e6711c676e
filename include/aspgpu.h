/*
 * aspgpu -- conflict-driven answer-set solving on one GB300 (sm_103a).
 *
 * C ABI of libaspgpu.so.  Every entry point takes plain host or device
 * pointers and sizes; no C++ or framework types cross this boundary.
 *
 * Method: Dovier, Formisano, Vella, "GPU-based parallelism for ASP-solving"
 * (arXiv 1909.01786).  A ground normal program is turned into completion
 * nogoods (Section 2), stored as a nogood store in device memory (Section 4),
 * and solved by conflict-driven nogood learning with ASP-computation
 * decisions (Section 2; Algorithm 1): propagation and checking of all
 * nogoods to a fixpoint (Section 4.1), conflict analysis from decision-level
 * dependency bitmaps (Section 4.2, Algorithm 4) or, as an option, by
 * resolution to the first UIP (Algorithm 3), backjumping, decisions, and
 * completion of the assignment.  Every step runs in this library's CUDA
 * kernels; the host only builds the nogood store and reads results.
 *
 * Conventions
 *  - Atoms are 0-based.  Rule r is  head[r] <- pos[pos_off[r]..pos_off[r+1]),
 *    not neg[neg_off[r]..neg_off[r+1]);  head[r] = -1 marks an integrity
 *    constraint (Section 1).  Repeated atoms in one body count once.
 *  - Solver variables: atoms 0..n_atoms-1, then for the j-th rule that has a
 *    head (rules ordered by head atom, ties in input order)
 *    b_j = n_atoms + 3j, t_j = n_atoms + 3j + 1, n_j = n_atoms + 3j + 2 (the
 *    auxiliary atoms b_r, t_r, n_r of Section 2).
 *  - Models are bitsets: row i of a model buffer holds ceil(n_atoms/64)
 *    uint64 words; bit (a mod 64) of word (a div 64) is atom a.
 *  - Return codes: ASP_OK or a negative ASP_E_*; asp_last_error() gives a
 *    message (thread-local).  Status values follow the SAT convention.
 *  - A program object is used by one host thread at a time; calls on
 *    different program objects may run concurrently on different streams.
 */
#ifndef ASPGPU_H
#define ASPGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ASP_OK 0
#define ASP_E_ARG (-1)       /* bad argument (null pointer, negative size, bad offsets) */
#define ASP_E_RANGE (-2)     /* atom id out of range, or too many variables */
#define ASP_E_OOM (-3)       /* device allocation failed */
#define ASP_E_CUDA (-4)      /* CUDA runtime error */
#define ASP_E_CAPACITY (-5)  /* caller's model buffer full; the models found so far are valid */
#define ASP_E_DEVICE (-6)    /* device-side error: learned-store overflow, barrier timeout, or
                                an inconsistent state met by resolution learning */
#define ASP_E_NODEVICE (-7)  /* no CUDA device / compiled kernels unavailable */

#define ASP_STATUS_UNKNOWN 0 /* budget exhausted before the answer was known */
#define ASP_STATUS_SAT 10    /* at least one answer set found */
#define ASP_STATUS_UNSAT 20  /* no (further) answer set exists */

#define ASP_HEUR_OCCURRENCE 0 /* static: occurrence count of the head (Section 4) */
#define ASP_HEUR_ACTIVITY 1   /* occurrence count plus activity bumped by conflicts */
#define ASP_HEUR_LEARNED 2    /* log1p(head occurrences) + log sigmoid(MLP logit) (not in the paper) */
#define ASP_HEUR_LEARNED_STATIC 3 /* the same score computed once per rule at load, with the
                                     search-state features at their values before the first
                                     decision: a learned static rule order (not in the paper) */
#define ASP_HEUR_JW 4         /* Jeroslow-Wang (Section 4): sum of 2^-|delta| over the nogoods
                                 delta holding Fb_r or F head(r), the clauses the decision
                                 Tb_r satisfies (computed at load) */
#define ASP_HEUR_VSIDS 5      /* decaying activity (Section 4 names activity among the decision
                                 heuristics; this form is not the paper's): each variable of a
                                 learned nogood bumps the rules it stands for (b_r, t_r, n_r its
                                 rule; an atom the rules with it as head) by an increment that
                                 grows by 1/0.95 per learned nogood; ties go to the head's
                                 occurrences, then to the lowest rule */

/* Shared-memory assignment view of each CTA during the propagate-and-check
 * sweep (Section 4.1; the layout is this implementation's, not the paper's).
 * PLAIN: 2 bits per variable, nogood literals name variables, variables
 * outside the view are read from global memory.  PACKED: 2 bits per
 * variable, every variable the CTA's nogoods name is in the view, and the
 * sweep reads a copy of the static store whose literals name view entries.
 * BYTES: as PACKED with one byte per variable. */
#define ASP_VIEW_AUTO 0       /* widest that fits: BYTES, PACKED, PLAIN */
#define ASP_VIEW_PLAIN 1
#define ASP_VIEW_PACKED 2
#define ASP_VIEW_BYTES 3

/* Conflict analysis (Section 4.2).  FWD: fwd-learning -- the learned
 * nogood is the decision literals of the levels in the OR of the conflict's
 * dependency bitmaps, and the search backjumps to the level below the
 * highest of them.  RES: resolution to the first UIP (Algorithm 3, the
 * analysis the paper compares fwd-learning against), run by one warp: the
 * learned nogood holds the first UIP of the conflict level and the literals
 * below it that the resolution reaches, and the search backjumps to the
 * highest level among the latter.  Root-level literals are left out of
 * either.  RES keeps a trail position, a stamp and a bit per variable (12
 * bytes per variable more). */
#define ASP_LEARN_FWD 0
#define ASP_LEARN_RES 1

/* Propagation rounds (Section 4.1; Algorithm 2 checks only the nogoods of
 * the literals assigned last).  FULL: every round sweeps every nogood.
 * NOGOODS: a round checks the nogoods holding a variable assigned in the
 * previous round, one lane per nogood from per-variable occurrence lists.
 * UNITS: a round sweeps the units of the static partition (32-nogood groups
 * of one bucket, as full sweeps take them) that hold a variable assigned in
 * the previous round; a claim marks them in a dirty bitmap for the next
 * round (single-program solving; a batch sweeps everything). */
#define ASP_FRONTIER_FULL 0
#define ASP_FRONTIER_NOGOODS 1
#define ASP_FRONTIER_UNITS 2
/* UNITS_CHAINED: as UNITS, and inside a round a claim also queues its CTA's
 * own units that hold the claimed variable, which later waves of the same
 * sweep check (up to three more waves; single-program solving). */
#define ASP_FRONTIER_UNITS_CHAINED 3

/* Backjump target of fwd-learning, with h the highest level in the
 * conflict's dependency bitmap.  H_MINUS_1: level h-1 (Algorithm 4's
 * reading).  ASSERTING: the second-highest level in the bitmap (1 if there
 * is none), where the learned nogood is already unit; it can jump further.
 * An overflowed bitmap (levels beyond deps_levels) always goes to h-1. */
#define ASP_BACKJUMP_H_MINUS_1 0
#define ASP_BACKJUMP_ASSERTING 1

#define ASP_MLP_FEATURES 16   /* inputs of the learned heuristic per candidate rule */
#define ASP_MLP_PARAMS 1153   /* W1[64][16], b1[64], w2[64], b2 */

typedef struct asp_prog asp_prog; /* opaque, owned by the library */

typedef struct {
    int32_t heuristic;        /* ASP_HEUR_* */
    int32_t deps_levels;      /* decision levels tracked exactly by the dependency
                                 bitmaps (Section 4.2); rounded up to a multiple of 64;
                                 deeper levels share one overflow bit. 0 = 4096 */
    int64_t conflict_budget;  /* stop with UNKNOWN after this many conflicts; 0 = none */
    int64_t time_budget_ms;   /* stop with UNKNOWN after this device time; 0 = none */
    int64_t learned_capacity; /* literals reserved for learned nogoods; 0 = automatic
                                 (8 x the static store, at least 2^24, at most 2^28) */
    int32_t grid_ctas;        /* CTAs of the persistent solver grid; 0 = one per SM */
    int32_t block_threads;    /* threads per CTA (multiple of 32, <= 768); 0 = 768 */
    void *cuda_stream;        /* cudaStream_t for all work of this program; NULL = default */
    /* device memory hooks; both NULL = cudaMalloc/cudaFree */
    void *(*dev_alloc)(size_t bytes, void *ctx);
    void (*dev_free)(void *ptr, size_t bytes, void *ctx);
    void *alloc_ctx;
    /* learned heuristic: ASP_MLP_PARAMS host floats, copied at load (used
       when heuristic = ASP_HEUR_LEARNED or ASP_HEUR_LEARNED_STATIC; stored as bf16) */
    const float *mlp_weights;
    /* record up to this many decisions per solve for asp_trace; 0 = none */
    int64_t trace_capacity;
    /* ASP_VIEW_*: the widest view allowed (a wider one than fits in shared
       memory falls back to the next narrower); 0 = ASP_VIEW_AUTO */
    int32_t view_mode;
    /* ASP_FRONTIER_*: which static nogoods a propagation round checks
       (Algorithm 2's frontier idea; the long and learned nogoods are checked
       every round, and rounds after backjumps sweep everything) */
    int32_t frontier;
    /* ASP_LEARN_*: conflict analysis */
    int32_t learning;
    /* ASP_BACKJUMP_*: target of fwd-learning's backjump (resolution
       learning always backjumps to its asserting level) */
    int32_t backjump;
    /* Luby restarts (not in the paper's experiments): after the i-th
       restart, restart again once luby(i+1) x restart_conflicts nogoods
       have been learned (1 1 2 1 1 2 4 ...) -- the backjump after that
       learned nogood goes to the root instead of its target; learned
       nogoods are kept.  0 = no restarts */
    int32_t restart_conflicts;
    /* conflicts analysed when a round finds several (Section 4.2 allows
       one or more): 1..4, 0 = 1.  The shortest conflicting nogood, then the
       shortest of each class of nogood ids mod 3, shorter first; each gives
       a learned nogood and the search backjumps to the lowest target */
    int32_t conflicts_per_round;
    /* 1: compact completion -- for a rule with an empty positive (negative)
       body, leave out {Tb_r, Ft_r} ({Tb_r, Fn_r}) and the literal Tt_r (Tn_r)
       of {Fb_r, Tt_r, Tn_r}; the unit nogood {Ft_r} ({Fn_r}) still sets t_r
       (n_r) at the root, so the variables and the answer sets are unchanged */
    int32_t compact;
} asp_options;

typedef struct {
    int64_t n_vars, n_atoms, n_rules_with_head;
    int64_t n_nogoods, n_literals;       /* static completion + constraint nogoods */
    int64_t n_unit_nogoods, n_long_nogoods;
    int64_t store_bytes;                 /* device bytes of the static nogood store */
    int64_t rounds;                      /* propagate-and-check sweeps (Section 4.1) */
    int64_t literal_checks;              /* literals read and classified by the sweeps */
    int64_t propagations, conflicts, decisions, completions;
    int64_t learned, learned_literals, loop_nogoods, models;
    int64_t max_level;
    int64_t ns_total, ns_sweep, ns_analysis, ns_decision, ns_stability; /* device time */
    int64_t ns_buckets, ns_learned, ns_barrier; /* CTA 0: static buckets, long and learned
                                                   nogoods, waiting at phase barriers */
    int64_t view_mode, batch_view_mode;         /* ASP_VIEW_* chosen for asp_solve and for
                                                   asp_solve_batch */
    int64_t ns_slowest_cta, ns_slowest_sweep;   /* sums over phases of the slowest CTA's time
                                                   before the phase barrier, and in the sweep */
    int64_t restarts;                           /* restarts (asp_options.restart_conflicts) */
    int64_t conflict_rounds;                    /* rounds that found a conflict; conflicts
                                                   counts every analysed one */
    int64_t nogood_visits;                      /* nogoods classified by the sweeps (the long
                                                   and learned ones every sweep, the bucket
                                                   ones in full sweeps; frontier rounds'
                                                   nogoods are not counted) */
    int64_t ns_slowest_long, ns_slowest_buckets; /* sums over sweeps of the slowest warp's time
                                                   (any CTA) on long and learned nogoods, and
                                                   on bucket units */
} asp_stats_t;

/* Default options (all zero except as documented above). */
void asp_default_options(asp_options *opt);

/* Build the completion nogoods of a ground normal program (Section 2) and
 * upload them.  Input arrays belong to the caller and are only read during
 * the call.  opt may be NULL.  On success *out owns device memory until
 * asp_free.  Errors: ASP_E_ARG, ASP_E_RANGE, ASP_E_OOM, ASP_E_CUDA,
 * ASP_E_NODEVICE. */
int asp_load_ground(int32_t n_atoms, int32_t n_rules, const int32_t *head,
                    const int64_t *pos_off, const int32_t *pos,
                    const int64_t *neg_off, const int32_t *neg,
                    const asp_options *opt, asp_prog **out);

/* Search for answer sets (Algorithm 1 on the device): up to max_models of
 * them (0 = all).  models: host buffer of models_cap rows (see Conventions).
 * Blocks until done.  status: ASP_STATUS_*; n_models: answer sets found.
 * Returns ASP_E_CAPACITY if more models were found than models_cap rows
 * (the first models_cap rows are written; *n_models is the count found). */
int asp_solve(asp_prog *p, int64_t max_models, uint64_t *models, int64_t models_cap,
              int64_t *n_models, int32_t *status);

/* Device-resident form of asp_solve: enqueues the whole search on the
 * program's stream and returns without synchronising.  d_models is a device
 * buffer of models_cap rows; d_result is a device int64[4] receiving
 * {status, n_models, error_code, 0}.  Sizes are as for asp_solve. */
int asp_solve_async(asp_prog *p, int64_t max_models, uint64_t *d_models, int64_t models_cap,
                    int64_t *d_result);

/* Solve n independent programs in one persistent launch, one CTA per program
 * at a time, taking programs from a device work queue largest first (not in
 * the paper, which solves one program per run).  progs[i] must have been
 * loaded with the same stream.  statuses[i], n_models[i] are host outputs;
 * models[i] (host, models_cap[i] rows) may be NULL when models_cap[i] is 0.
 * Same as asp_batch_create (configuration 0) + asp_batch_run +
 * asp_batch_free. */
int asp_solve_batch(int32_t n, asp_prog *const *progs, int64_t max_models_each,
                    int32_t *statuses, int64_t *n_models, uint64_t *const *models,
                    const int64_t *models_cap);

/* A batch prepared for repeated solving (not in the paper). */
typedef struct asp_batch asp_batch;

#define ASP_BATCH_AUTOTUNE (-1)   /* let the autotuner choose the configuration */

/* Prepare repeated batched solving of n loaded programs: uploads one
 * descriptor per program, chooses the kernel configuration and the
 * propagation schedule, and captures the launch (queue reset + batch
 * kernel) in a CUDA graph.  Configurations: 0 = 256 threads per CTA, 3 CTAs
 * per SM; 1 = 128 threads, 6 per SM (twice the programs in flight, smaller
 * shared-memory views).  With an explicit configuration each program keeps
 * its own frontier option.  config = ASP_BATCH_AUTOTUNE tries every schedule
 * -- each configuration with full sweeps and, where the programs are small
 * enough to have the lists (about 20k atoms at 4 rules per atom), with the
 * frontier by units -- once on a sample of up to 256 programs spread over
 * the queue (each with at most 8 conflicts and 0.5 s of device time), and
 * keeps the one with the lowest device time per program (the trial solves
 * change nothing but the programs' last results).  models_cap may be NULL
 * (no models kept).  The programs must stay loaded until asp_batch_free.
 * Errors: ASP_E_ARG, ASP_E_OOM, ASP_E_CUDA. */
int asp_batch_create(int32_t n, asp_prog *const *progs, int64_t max_models_each, const int64_t *models_cap,
                     int32_t config, asp_batch **out);

/* Replay the captured launch: every program of the batch is solved from
 * scratch.  Outputs and errors as asp_solve_batch (models[i] may be NULL
 * when the capacity given at creation is 0). */
int asp_batch_run(asp_batch *b, int32_t *statuses, int64_t *n_models, uint64_t *const *models);

/* The configuration in use (0 or 1), its threads per CTA, the grid, the
 * propagation schedule (ASP_FRONTIER_UNITS for programs with unit lists, or
 * ASP_FRONTIER_FULL), and trial_ns (host double[4]): the autotuner's device
 * time per program of configurations 0 and 1 with full sweeps, then 0 and 1
 * with the unit frontier (ns; 0 if not tried, < 0 if it could not run); any
 * output may be NULL. */
int asp_batch_info(const asp_batch *b, int32_t *config, int32_t *block_threads, int32_t *grid,
                   int32_t *frontier, double *trial_ns);

/* Release the batch's descriptors, graph and stream (not the programs). */
void asp_batch_free(asp_batch *b);

/* Counters of the last solve on this program (device time in ns). */
int asp_stats(const asp_prog *p, asp_stats_t *out);

/* Release all device memory of the program. */
void asp_free(asp_prog *p);

/* Message of the last error on this host thread ("" if none). */
const char *asp_last_error(void);

/* ---- test and measurement entry points ---------------------------------
 * Unit propagation to fixpoint alone (Section 4.1, propagate-and-check):
 * partial[v] in {1 true, -1 false, 0 unassigned} over all solver variables
 * (host, n_vars entries), taken as root-level input; the static nogoods are
 * then swept until no nogood is unit.  closure (host, n_vars) receives the
 * result; *conflict = 1 if some nogood became violated (closure is then the
 * state at that point).  The input must not itself assign a variable twice;
 * it may violate nogoods. */
int asp_debug_propagate(asp_prog *p, const int8_t *partial, int8_t *closure, int32_t *conflict);

/* Propagate-and-check sweeps over the whole static store against the
 * current device assignment, without claiming anything (used to time the
 * sweep in isolation): one launch loads each CTA's shared-memory view once,
 * then makes `passes` full passes.  Enqueued on the program's stream. */
int asp_sweep(asp_prog *p, int32_t passes);

/* Copy of the state after the last solve or debug call, for consistency
 * checks: trail (n_trail variables in assignment order), per variable
 * level (int32, 0 = unassigned), reason (uint32 nogood id, 0xFFFFFFFF =
 * decision, 0xFFFFFFFE = completion step, 0xFFFFFFFD = input) and the first
 * deps_words uint64 words of each variable's dependency bitmap.  Host
 * buffers; any may be NULL.  *n_trail receives the trail length. */
int asp_debug_state(asp_prog *p, int32_t *trail, int64_t *n_trail, int32_t *level,
                    uint32_t *reason, uint64_t *deps, int32_t deps_words);

/* The last conflict analysis of the last solve, for consistency checks.
 * info (host int64[6]): {conflicting nogood id, trail length at the conflict
 * (claims of the conflict round included), learned nogood id, its length,
 * backjump target, level resolved at (ASP_LEARN_RES; 0 for ASP_LEARN_FWD)}.
 * Length 0 and target 0: no conflict was analysed.  Length 0 and target
 * t > 0: the resolution found the state inconsistent (the solve then ends
 * with ASP_E_DEVICE) -- t numbers the failed check (1 literal outside the
 * variables, 2 unassigned, 3 above the conflict level, 4 trail position
 * outside its level, 5 nogood without end, 6/7 marked literals and count
 * disagree, 8 trail entry outside the variables, 9 decision or input
 * resolved upon, 10 empty level) and info[2] holds the variable or value
 * involved.  trail (host, may be NULL) receives
 * up to trail_cap entries of the trail at that point as literals
 * (var << 1 | sign, sign 1 = F), in assignment order.  When the solve
 * stopped on its conflict budget right after that analysis (before the
 * backjump), levels and reasons from asp_debug_state describe the same
 * assignment. */
int asp_debug_last_conflict(asp_prog *p, int64_t *info, int32_t *trail, int64_t trail_cap);

/* Literals of nogood `id` (a reason or learned id) as (var << 1 | sign),
 * sign 1 = F; returns the length, writes at most cap literals. */
int64_t asp_debug_nogood(asp_prog *p, uint32_t id, int32_t *lits, int64_t cap);

/* Ids of the nogoods learned by the last solve, in the order they were
 * added (Algorithm 1's learned set: fwd-learning or resolution nogoods,
 * loop nogoods of the stability step, and the blocking nogoods of the
 * answer sets found); each id is an offset in the literal store accepted
 * by asp_debug_nogood.  ids: host buffer of cap entries (may be NULL when
 * cap is 0).  Returns the number learned (possibly more than cap) or a
 * negative ASP_E_*. */
int64_t asp_debug_learned(asp_prog *p, uint32_t *ids, int64_t cap);

/* The completion nogoods (Section 2: the nogoods of each rule's body
 * definition b_j <-> t_j & n_j, t_j <-> B+, n_j <-> not B-, head <- b_j, each
 * atom's support nogood {Tp} u {Fb_j : head(j) = p}, one nogood per
 * constraint) exactly as asp_load_ground builds them on the host, computed
 * on the host alone (no device is touched, so it runs on machines without a
 * GPU).  The program arguments are those of asp_load_ground; compact != 0
 * takes the compact completion of asp_options.compact.  Variables are the
 * library's: atoms 0..n_atoms-1, then b_j, t_j, n_j = n_atoms + 3j + 0/1/2
 * for the headed rules j ordered by head atom (ties in input order).
 *   n_vars, n_nogoods, n_literals  outputs (required)
 *   off   host int64[n_nogoods + 1]: nogood i is lits[off[i] .. off[i+1])
 *   lits  host int32[lits_cap]: literals (var << 1 | sign), sign 1 = F
 * Pass off = lits = NULL to read the counts first.  Order: the nogoods of
 * length 2..15 by length (an atom's rule nogoods and its own nogood
 * together, atom by atom, then the constraints), then the longer ones, the
 * unit nogoods, and one empty nogood per empty constraint.  Returns ASP_OK,
 * ASP_E_ARG / ASP_E_RANGE as asp_load_ground does, or ASP_E_CAPACITY if
 * lits_cap < n_literals.  Caller owns every buffer. */
int asp_debug_completion(int32_t n_atoms, int32_t n_rules, const int32_t *head,
                         const int64_t *pos_off, const int32_t *pos,
                         const int64_t *neg_off, const int32_t *neg, int32_t compact,
                         int64_t *n_vars, int64_t *n_nogoods, int64_t *n_literals,
                         int64_t *off, int32_t *lits, int64_t lits_cap);

/* The static decision scores of the headed rules (Section 4, Decision:
 * occurrences and Jeroslow-Wang), as asp_load_ground computes them on the
 * host, without a device.  For rule j of the library's order (headed rules
 * by head atom, ties in input order): rule_index[j] = its input index,
 * score_occ[j] = occurrences of its head atom in the completion's literals
 * (heuristic ASP_HEUR_OCCURRENCE), score_jw[j] = sum of 2^(16 - |delta|)
 * over the nogoods delta holding F b_j, plus the same over those holding
 * F head(j) (heuristic ASP_HEUR_JW; nogoods longer than 16 add 0; saturates
 * at 2^31 - 1).  n_headed (required) receives the number of headed rules;
 * any of the three arrays may be NULL, the others hold cap entries.
 * Returns ASP_OK, the errors of asp_load_ground's argument checks, or
 * ASP_E_CAPACITY if cap < n_headed. */
int asp_debug_rule_scores(int32_t n_atoms, int32_t n_rules, const int32_t *head,
                          const int64_t *pos_off, const int32_t *pos,
                          const int64_t *neg_off, const int32_t *neg, int32_t compact,
                          int32_t *n_headed, int32_t *rule_index, uint32_t *score_occ,
                          uint32_t *score_jw, int64_t cap);

/* Test-only failure injection at the grid barrier of asp_solve (the
 * persistent kernel's phase barrier, Algorithm 1's steps run between them):
 * CTA stall_cta of the solver grid does not arrive at the first phase
 * barrier -- it waits on a flag that nothing sets -- and every CTA gives up
 * on a barrier after wait_limit_ms.  The solve then returns ASP_E_DEVICE and
 * the CUDA context stays usable; the stalled CTA's own wait ends when
 * another CTA has given up (or after 3 x wait_limit_ms).  stall_cta < 0 and
 * wait_limit_ms <= 0 restore the defaults (no stall, 20 s).  Applies to
 * later solves of p.  Errors: ASP_E_ARG. */
int asp_debug_barrier(asp_prog *p, int32_t stall_cta, int32_t wait_limit_ms);

/* Test-only failure injection on the host: the nth device allocation the
 * library makes from now on (any program, any thread) fails as if the
 * allocator had no memory, so the call that needed it returns ASP_E_OOM.
 * nth = 0 switches it off.  Errors: ASP_E_ARG. */
int asp_debug_fail_alloc(int64_t nth);

/* The compute capability the solve kernel was compiled for
 * (binary_version, 103 for sm_103a) and its PTX version, as the CUDA
 * runtime reports them for the current device; either output may be NULL.
 * Errors: ASP_E_NODEVICE, ASP_E_CUDA. */
int asp_build_info(int32_t *binary_version, int32_t *ptx_version);

/* ---- learned decision heuristic (not in the paper) ------------------------
 * Decision traces of the last solve, for training: at every Decision step
 * about one applicable rule in eight is sampled, giving one row of
 * ASP_MLP_FEATURES floats (8 static features of the rule, log1p activity,
 * B- atoms unassigned and false, level/64, log1p conflicts, assigned
 * fraction, 0, 0) and a label: 1 if the rule's body holds in the first
 * answer set the search found, 0 if not, -1 if no answer set was found.
 * rules (may be NULL) receives each row's rule index j (solver numbering,
 * see Conventions).  Host buffers of cap rows; returns the number of rows
 * (at most trace_capacity), or a negative ASP_E_*. */
int64_t asp_trace(asp_prog *p, float *features, int32_t *labels, int32_t *rules, int64_t cap);

/* Train the heuristic's MLP (16 -> 64 ReLU -> 1, logistic output) on the
 * device: minibatches of 4096, SGD with momentum 0.9, binary cross-entropy.
 * features: host [n][ASP_MLP_FEATURES]; labels: host [n] in {0, 1};
 * weights: host [ASP_MLP_PARAMS], initial values in, trained values out.
 * Blocks until done.  Uses the current device and allocates its own
 * buffers. */
int asp_train_mlp(const float *features, const float *labels, int64_t n, int32_t epochs,
                  float learning_rate, float *weights);

/* Scores of n feature rows under the given weights, computed on the device
 * exactly as the Decision step does (weights rounded to bf16, fp32
 * accumulation).  Host buffers: features [n][ASP_MLP_FEATURES], scores [n]. */
int asp_mlp_score(const float *weights, const float *features, int64_t n, float *scores);

/* ---- allocation-free propagation ---------------------------------------
 * The paper has no counterpart of this entry point; it exists for callers
 * that cannot allocate device memory where they need propagation --
 * real-time loops that must not enter the allocator (an allocation can
 * block on the driver or force a synchronising release of cached blocks),
 * and processes whose device memory is handed out up front by a pool or a
 * framework that owns all of it.  It computes the same closure as
 * asp_debug_propagate (unit propagation of a root-level partial assignment
 * to fixpoint over the program's nogoods) but keeps all of its working
 * memory in one static device array inside the library: at most 2^20
 * solver variables (512 KB of 4-bit codes plus 256 B of counters), held by
 * every GPU that loads the library until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   p          a program loaded earlier with asp_load_ground (read only)
 *   d_partial  device int8[n_vars]: 1 true, -1 false, 0 unassigned
 *   d_closure  device int8[n_vars] output: 1 / -1 / 0 (2 marks a variable
 *              both values were claimed for, only after a conflict)
 *   d_conflict device int32 output: 1 if a nogood became violated,
 *              -1 on a device-side barrier timeout, else 0
 * The work is enqueued on the program's stream; the call returns without
 * synchronising.  The device the program was loaded on must be the current
 * device.  Returns ASP_E_CAPACITY if the program has more than 2^20
 * variables, ASP_E_ARG on null pointers or when another device is current,
 * ASP_E_CUDA on a CUDA error.  The first call on a device looks up the
 * device address of the static array (cudaGetSymbolAddress) and the
 * kernel's occupancy; make that first call before any stream capture.
 * Every call shares the one array: calls that overlap on the GPU (other
 * streams, other host threads) race on it and give wrong results.  Each call clears the counters it needs at zero. */
int asp_propagate_noalloc(const asp_prog *p, const int8_t *d_partial, int8_t *d_closure,
                          int32_t *d_conflict);

#ifdef __cplusplus
}
#endif
#endif /* ASPGPU_H */
