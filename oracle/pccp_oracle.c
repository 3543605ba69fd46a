/*
 * pccp_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, sequential CPU oracle for the propagate-and-search method of
 * "A Variant of Concurrent Constraint Programming on GPU" (Talbot, Pinel,
 * Bouvry, AAAI 2022).  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code; the product path never
 * does.  It shares no code, header or table with the CUDA library.
 *
 * All values are int64 so no intermediate can overflow for the int32 models
 * the library accepts.
 *
 * What it computes (with the passages followed):
 *  - Store: a product of interval lattices IZ = ZInc x ZDec (Sec. 2), one
 *    (lb, ub) pair per variable; a tell joins (lb <- max, ub <- min).
 *  - Constraints are compiled to guarded commands (GNF, Sec. 3, Prop. 3):
 *      temporal x + d <= y       : the [[x + y <= c]] compilation of Sec. 2
 *                                  with y' = -y, c = -d  (2 commands)
 *      reified b <=> (A and B),  A: x <= y, B: y < x + d
 *                                : the four asks of [[phi <=> psi]] (Sec. 2),
 *                                  with [[A and B]] = [[A]] || [[B]] (11 commands)
 *      linear  sum a_k x_k <= c  : one bound tell per term from the minimum of
 *                                  the other terms (the resource-sum compilation
 *                                  of Sec. 2, generalised to any sign; the term
 *                                  itself is left out of the sum)
 *  - propagate: the least fixed point above the input store of the join of
 *    all guarded commands (Theorem 1), computed by sweeps in one of several
 *    fair orders (seq P of Prop. 2; the fair schedules of Def. 4):
 *      forward Gauss-Seidel, reverse, a fresh random permutation per sweep,
 *      or Jacobi (every command reads the sweep's starting store, Sec. 3's D).
 *    Failure (an empty interval, the top of the lattice; Sec. 5) is checked
 *    after every tell.
 *  - solve: depth-first branch and bound.  Every node's store is
 *    fix(root join path-decisions join {ub(obj) <= best-1}); a node is every
 *    store propagated.  Branching: lowest-index unfixed branch variable
 *    (input order) or smallest interval first (first-fail, ties to the lower
 *    index); split [l,u] at m = l + (u-l)/2, left child ub <= m first, right
 *    child lb >= m+1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;

/* Plain-data model, filled by the Python wrapper from numpy arrays. */
typedef struct {
  int32_t n_vars;
  const i64* lb0;
  const i64* ub0;
  int32_t n_temporal;
  const int32_t* t_x;
  const int32_t* t_y;
  const i64* t_d;
  int32_t n_reified;
  const int32_t* r_b;
  const int32_t* r_x;
  const int32_t* r_y;
  const i64* r_d;
  int32_t n_linear;
  const i64* l_c;
  const int32_t* l_off; /* n_linear + 1 offsets into l_var/l_coef */
  const int32_t* l_var;
  const i64* l_coef;
  int32_t objective; /* variable to minimise, or -1 */
  int32_t n_branch;
  const int32_t* branch;
} om_model;

enum { OM_FIXPOINT = 0, OM_FAILED = 1, OM_NONTERMINATING = 2 };
enum { OM_FORWARD = 0, OM_REVERSE = 1, OM_RANDOM = 2, OM_JACOBI = 3 };

#define OM_NO_TELL 0
#define OM_TELL_LB 1
#define OM_TELL_UB 2

/* One tell produced by a guarded command: join value into lb or ub of var. */
typedef struct {
  int kind;
  int32_t var;
  i64 value;
} om_tell;

#define REIFIED_COMMANDS 11

static i64 floor_div(i64 a, i64 b) { /* b > 0 */
  i64 q = a / b;
  if ((a % b != 0) && (a < 0)) q -= 1;
  return q;
}

static i64 ceil_div(i64 a, i64 b) { /* b > 0 */
  return -floor_div(-a, b);
}

int64_t om_command_count(const om_model* m) {
  return 2 * (int64_t)m->n_temporal + (int64_t)REIFIED_COMMANDS * m->n_reified +
         (int64_t)m->l_off[m->n_linear];
}

/* Temporal x + d <= y as [[x + y' <= c]] with y' = -y, c = -d:
 *   x  <- (bot, c - lb(y'))  i.e.  ub(x) <= ub(y) - d
 *   y' <- (bot, c - lb(x))   i.e.  lb(y) >= lb(x) + d                      */
static om_tell temporal_command(const om_model* m, const i64* lb, const i64* ub, int32_t t,
                                int which) {
  om_tell r;
  int32_t x = m->t_x[t], y = m->t_y[t];
  i64 d = m->t_d[t];
  if (which == 0) {
    r.kind = OM_TELL_UB; r.var = x; r.value = ub[y] - d;
  } else {
    r.kind = OM_TELL_LB; r.var = y; r.value = lb[x] + d;
  }
  return r;
}

/* Reified b <=> (A and B) with A: x <= y and B: y <= x + d - 1.
 *   entailed(A)    : ub x <= lb y          entailed(B)    : ub y <= lb x + d - 1
 *   entailed(not A): lb x >= ub y + 1      entailed(not B): lb y >= ub x + d
 * Commands (the four asks of [[phi <=> psi]] with phi = (b >= 1)):
 *   0-3  if lb b >= 1            : [[A]] = {ub x <= ub y, lb y >= lb x},
 *                                  [[B]] = {ub y <= ub x + d - 1, lb x >= lb y - d + 1}
 *   4    if entailed(A and B)    : lb b >= 1
 *   5    if entailed(not A)      : ub b <= 0
 *   6    if entailed(not B)      : ub b <= 0
 *   7-8  if ub b <= 0 and entailed(A): [[not B]] = {lb y >= lb x + d, ub x <= ub y - d}
 *   9-10 if ub b <= 0 and entailed(B): [[not A]] = {lb x >= lb y + 1, ub y <= ub x - 1}  */
static om_tell reified_command(const om_model* m, const i64* lb, const i64* ub, int32_t r,
                               int which) {
  om_tell t;
  int32_t b = m->r_b[r], x = m->r_x[r], y = m->r_y[r];
  i64 d = m->r_d[r];
  int ent_A = ub[x] <= lb[y];
  int ent_B = ub[y] <= lb[x] + d - 1;
  int ent_notA = lb[x] >= ub[y] + 1;
  int ent_notB = lb[y] >= ub[x] + d;
  t.kind = OM_NO_TELL; t.var = 0; t.value = 0;
  switch (which) {
    case 0: if (lb[b] >= 1) { t.kind = OM_TELL_UB; t.var = x; t.value = ub[y]; } break;
    case 1: if (lb[b] >= 1) { t.kind = OM_TELL_LB; t.var = y; t.value = lb[x]; } break;
    case 2: if (lb[b] >= 1) { t.kind = OM_TELL_UB; t.var = y; t.value = ub[x] + d - 1; } break;
    case 3: if (lb[b] >= 1) { t.kind = OM_TELL_LB; t.var = x; t.value = lb[y] - d + 1; } break;
    case 4: if (ent_A && ent_B) { t.kind = OM_TELL_LB; t.var = b; t.value = 1; } break;
    case 5: if (ent_notA) { t.kind = OM_TELL_UB; t.var = b; t.value = 0; } break;
    case 6: if (ent_notB) { t.kind = OM_TELL_UB; t.var = b; t.value = 0; } break;
    case 7: if (ub[b] <= 0 && ent_A) { t.kind = OM_TELL_LB; t.var = y; t.value = lb[x] + d; } break;
    case 8: if (ub[b] <= 0 && ent_A) { t.kind = OM_TELL_UB; t.var = x; t.value = ub[y] - d; } break;
    case 9: if (ub[b] <= 0 && ent_B) { t.kind = OM_TELL_LB; t.var = x; t.value = lb[y] + 1; } break;
    case 10: if (ub[b] <= 0 && ent_B) { t.kind = OM_TELL_UB; t.var = y; t.value = ub[x] - 1; } break;
    default: break;
  }
  return t;
}

/* Linear sum_k a_k x_k <= c, command for term k of row l:
 *   S_k = sum_{j != k} min over the box of a_j x_j  (a_j lb x_j if a_j > 0,
 *         a_j ub x_j otherwise),  slack = c - S_k
 *   a_k > 0: ub x_k <= floor(slack / a_k);   a_k < 0: lb x_k >= ceil(slack / a_k) */
static om_tell linear_command(const om_model* m, const i64* lb, const i64* ub, int32_t l,
                              int32_t k) {
  om_tell t;
  i64 others = 0;
  for (int32_t j = m->l_off[l]; j < m->l_off[l + 1]; ++j) {
    if (j == k) continue;
    i64 a = m->l_coef[j];
    int32_t v = m->l_var[j];
    others += (a > 0) ? a * lb[v] : a * ub[v];
  }
  i64 slack = m->l_c[l] - others;
  i64 a = m->l_coef[k];
  t.var = m->l_var[k];
  if (a > 0) {
    t.kind = OM_TELL_UB;
    t.value = floor_div(slack, a);
  } else if (a < 0) {
    t.kind = OM_TELL_LB;
    /* a x <= slack with a < 0  <=>  x >= slack / a  <=>  x >= ceil(slack / a),
     * and slack / a = (-slack) / (-a) with -a > 0 */
    t.value = ceil_div(-slack, -a);
  } else {
    t.kind = OM_NO_TELL;
    t.value = 0;
  }
  return t;
}

/* Guarded command number g in GNF order: temporal, reified, linear terms. */
static om_tell command(const om_model* m, const i64* lb, const i64* ub, int64_t g) {
  int64_t nt = 2 * (int64_t)m->n_temporal;
  if (g < nt) return temporal_command(m, lb, ub, (int32_t)(g / 2), (int)(g % 2));
  g -= nt;
  int64_t nr = (int64_t)REIFIED_COMMANDS * m->n_reified;
  if (g < nr)
    return reified_command(m, lb, ub, (int32_t)(g / REIFIED_COMMANDS),
                           (int)(g % REIFIED_COMMANDS));
  g -= nr;
  /* term g belongs to the row l with l_off[l] <= g < l_off[l+1] */
  int32_t l = 0;
  while (m->l_off[l + 1] <= g) ++l;
  return linear_command(m, lb, ub, l, (int32_t)g);
}

/* Join a tell into the store.  Returns 1 if the store changed. */
static int join(i64* lb, i64* ub, om_tell t) {
  if (t.kind == OM_TELL_LB && t.value > lb[t.var]) { lb[t.var] = t.value; return 1; }
  if (t.kind == OM_TELL_UB && t.value < ub[t.var]) { ub[t.var] = t.value; return 1; }
  return 0;
}

static int empty_at(const i64* lb, const i64* ub, int32_t v) { return lb[v] > ub[v]; }

static uint64_t splitmix_next(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/*
 * om_propagate: lb/ub hold the input store (n_vars each) and are overwritten
 * with the least fixed point above (input join root).  Returns OM_FIXPOINT or
 * OM_FAILED (store contents then unspecified).  *sweeps gets the number of
 * sweeps run.  max_sweeps bounds the loop (OM_NONTERMINATING if hit).
 */
int om_propagate(const om_model* m, i64* lb, i64* ub, int order, uint64_t seed,
                 int64_t max_sweeps, int64_t* sweeps) {
  int64_t nc = om_command_count(m);
  int64_t* perm = NULL;
  i64 *lb_start = NULL, *ub_start = NULL;
  int status = OM_FIXPOINT;
  int64_t s = 0;
  for (int32_t v = 0; v < m->n_vars; ++v) {
    if (m->lb0[v] > lb[v]) lb[v] = m->lb0[v];
    if (m->ub0[v] < ub[v]) ub[v] = m->ub0[v];
  }
  for (int32_t v = 0; v < m->n_vars; ++v)
    if (empty_at(lb, ub, v)) { if (sweeps) *sweeps = 0; return OM_FAILED; }
  if (order == OM_RANDOM || order == OM_REVERSE) {
    perm = (int64_t*)malloc(sizeof(int64_t) * (nc > 0 ? nc : 1));
    for (int64_t i = 0; i < nc; ++i) perm[i] = (order == OM_REVERSE) ? nc - 1 - i : i;
  }
  if (order == OM_JACOBI) {
    lb_start = (i64*)malloc(sizeof(i64) * (m->n_vars > 0 ? m->n_vars : 1));
    ub_start = (i64*)malloc(sizeof(i64) * (m->n_vars > 0 ? m->n_vars : 1));
  }
  uint64_t rng = seed;
  for (;;) {
    int changed = 0;
    if (s >= max_sweeps) { status = OM_NONTERMINATING; break; }
    ++s;
    if (order == OM_RANDOM) { /* Fisher-Yates, a fresh fair order per sweep */
      for (int64_t i = nc - 1; i > 0; --i) {
        int64_t j = (int64_t)(splitmix_next(&rng) % (uint64_t)(i + 1));
        int64_t tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
      }
    }
    if (order == OM_JACOBI) {
      memcpy(lb_start, lb, sizeof(i64) * m->n_vars);
      memcpy(ub_start, ub, sizeof(i64) * m->n_vars);
      for (int64_t g = 0; g < nc; ++g) {
        om_tell t = command(m, lb_start, ub_start, g);
        if (join(lb, ub, t)) {
          changed = 1;
          if (empty_at(lb, ub, t.var)) { status = OM_FAILED; goto done; }
        }
      }
    } else {
      for (int64_t i = 0; i < nc; ++i) {
        int64_t g = perm ? perm[i] : i;
        om_tell t = command(m, lb, ub, g);
        if (join(lb, ub, t)) {
          changed = 1;
          if (empty_at(lb, ub, t.var)) { status = OM_FAILED; goto done; }
        }
      }
    }
    if (!changed) break;
  }
done:
  free(perm);
  free(lb_start);
  free(ub_start);
  if (sweeps) *sweeps = s;
  return status;
}

/* Apply one guarded command once; exported for the per-command stability
 * and monotonicity tests. Returns the tell kind; *var / *value get the tell. */
int om_command(const om_model* m, const i64* lb, const i64* ub, int64_t g, int32_t* var,
               i64* value) {
  om_tell t = command(m, lb, ub, g);
  *var = t.var;
  *value = t.value;
  return t.kind;
}

/* ------------------------------------------------------------------ solve */

enum { OM_OPTIMISE = 0, OM_COUNT_ALL = 1 };
enum { OM_INPUT_ORDER = 0, OM_FIRST_FAIL = 1 };
enum { OM_RES_OPTIMAL = 0, OM_RES_INFEASIBLE = 1, OM_RES_LIMIT = 2 };

typedef struct {
  int32_t mode;
  int32_t strategy;
  int64_t node_limit; /* <= 0: none */
  i64 obj_ub;         /* inclusive bound told on the objective at every node */
} om_solve_opts;

typedef struct {
  int32_t status;
  int32_t has_solution;
  i64 objective;
  int64_t nodes;
  int64_t fails;
  int64_t solutions;
  int64_t sweeps;
  int32_t max_depth;
} om_solve_result;

typedef struct {
  const om_model* m;
  const om_solve_opts* o;
  om_solve_result* r;
  i64* witness; /* lb of the best (or first) solution, n_vars */
  i64 best;     /* best objective so far */
  int stop;
  /* decision path: var, kind (OM_TELL_UB left / OM_TELL_LB right), value */
  int32_t* dvar;
  int* dkind;
  i64* dval;
  i64* lb;
  i64* ub;
  int32_t cap;
  int64_t sweep_cap;
  /* optional record of every node in depth-first preorder (NULL: none) */
  int64_t* trace;
  int64_t trace_cap;
  int64_t trace_n;
} om_search;

/* Outcome of a node in the search trace. */
enum { OM_NODE_FAILED = 0, OM_NODE_SOLUTION = 1, OM_NODE_BRANCH = 2 };
#define OM_TRACE_FIELDS 6

/* Append one node to the trace: its depth, the decision that created it
 * (variable, side 0 = left ub <= value / 1 = right lb >= value, value; the
 * root has variable -1), its outcome and, for a branching node, the
 * variable chosen (else -1). */
static void trace_node(om_search* s, int32_t depth, int outcome, int32_t chosen) {
  if (!s->trace) return;
  if (s->trace_n < s->trace_cap) {
    int64_t* t = s->trace + OM_TRACE_FIELDS * s->trace_n;
    t[0] = depth;
    t[1] = depth > 0 ? s->dvar[depth - 1] : -1;
    t[2] = depth > 0 ? (s->dkind[depth - 1] == OM_TELL_UB ? 0 : 1) : -1;
    t[3] = depth > 0 ? s->dval[depth - 1] : 0;
    t[4] = outcome;
    t[5] = chosen;
  }
  s->trace_n += 1;
}

/* Branching variable (index into the store) or -1 if all branch vars fixed. */
static int32_t select_var(const om_model* m, int strategy, const i64* lb, const i64* ub) {
  int32_t best = -1;
  i64 best_w = 0;
  for (int32_t k = 0; k < m->n_branch; ++k) {
    int32_t v = m->branch[k];
    i64 w = ub[v] - lb[v];
    if (w <= 0) continue;
    if (strategy == OM_INPUT_ORDER) return v;
    if (best < 0 || w < best_w) { best = v; best_w = w; }
  }
  return best;
}

static void dfs(om_search* s, int32_t depth) {
  const om_model* m = s->m;
  if (s->stop) return;
  if (s->o->node_limit > 0 && s->r->nodes >= s->o->node_limit) { s->stop = 2; return; }
  s->r->nodes += 1;
  if (depth > s->r->max_depth) s->r->max_depth = depth;
  /* node store = root join path decisions join objective bound */
  for (int32_t v = 0; v < m->n_vars; ++v) { s->lb[v] = m->lb0[v]; s->ub[v] = m->ub0[v]; }
  for (int32_t i = 0; i < depth; ++i) {
    om_tell t; t.kind = s->dkind[i]; t.var = s->dvar[i]; t.value = s->dval[i];
    join(s->lb, s->ub, t);
  }
  if (m->objective >= 0) {
    i64 bound = s->o->obj_ub;
    if (s->o->mode == OM_OPTIMISE && s->r->has_solution && s->best - 1 < bound) bound = s->best - 1;
    if (bound < s->ub[m->objective]) s->ub[m->objective] = bound;
  }
  int64_t sw = 0;
  int st = om_propagate(m, s->lb, s->ub, OM_FORWARD, 0, s->sweep_cap, &sw);
  s->r->sweeps += sw;
  if (st == OM_NONTERMINATING) { s->stop = 4; return; }
  if (st != OM_FIXPOINT) {
    s->r->fails += 1;
    trace_node(s, depth, OM_NODE_FAILED, -1);
    return;
  }
  int32_t v = select_var(m, s->o->strategy, s->lb, s->ub);
  trace_node(s, depth, v < 0 ? OM_NODE_SOLUTION : OM_NODE_BRANCH, v);
  if (v < 0) {
    s->r->solutions += 1;
    i64 obj = (m->objective >= 0) ? s->lb[m->objective] : 0;
    int record = 0;
    if (s->o->mode == OM_OPTIMISE) record = 1; /* every solution found improves */
    else if (!s->r->has_solution) record = 1; /* count-all: keep the first */
    if (record) {
      s->best = obj;
      s->r->objective = obj;
      memcpy(s->witness, s->lb, sizeof(i64) * m->n_vars);
    }
    s->r->has_solution = 1;
    if (s->o->mode == OM_OPTIMISE && m->objective < 0) s->stop = 1; /* satisfaction */
    return;
  }
  if (depth + 1 > s->cap) { s->stop = 3; return; }
  i64 l = s->lb[v], u = s->ub[v];
  i64 mid = l + (u - l) / 2;
  s->dvar[depth] = v; s->dkind[depth] = OM_TELL_UB; s->dval[depth] = mid;
  dfs(s, depth + 1);
  if (s->stop) return;
  s->dvar[depth] = v; s->dkind[depth] = OM_TELL_LB; s->dval[depth] = mid + 1;
  dfs(s, depth + 1);
}

/* Returns 0 on success, -1 if the decision stack capacity was exceeded, -2 if
 * a propagation ran past its sweep bound (cannot happen for a correct
 * oracle; it turns a broken build into an error instead of a hang).
 * trace (may be NULL): room for trace_cap nodes of OM_TRACE_FIELDS int64
 * each (trace_node), filled in depth-first preorder; *trace_n (if not NULL)
 * receives the number of nodes, which may exceed trace_cap. */
int om_solve_traced(const om_model* m, const om_solve_opts* o, om_solve_result* r, i64* witness,
                    int64_t* trace, int64_t trace_cap, int64_t* trace_n) {
  om_search s;
  memset(r, 0, sizeof(*r));
  s.m = m; s.o = o; s.r = r; s.witness = witness; s.best = 0; s.stop = 0;
  s.trace = trace; s.trace_cap = trace ? trace_cap : 0; s.trace_n = 0;
  /* each decision strictly narrows one branch variable's interval; 64 per
   * variable bounds the depth for any int64 interval */
  s.cap = 64 * (m->n_branch > 0 ? m->n_branch : 1) + 1;
  /* each changing sweep narrows a bound by >= 1: width of the root box + 2 */
  s.sweep_cap = 2;
  for (int32_t v = 0; v < m->n_vars; ++v) s.sweep_cap += m->ub0[v] - m->lb0[v] + 1;
  s.dvar = (int32_t*)malloc(sizeof(int32_t) * s.cap);
  s.dkind = (int*)malloc(sizeof(int) * s.cap);
  s.dval = (i64*)malloc(sizeof(i64) * s.cap);
  s.lb = (i64*)malloc(sizeof(i64) * (m->n_vars > 0 ? m->n_vars : 1));
  s.ub = (i64*)malloc(sizeof(i64) * (m->n_vars > 0 ? m->n_vars : 1));
  dfs(&s, 0);
  int rc = (s.stop == 3) ? -1 : (s.stop == 4) ? -2 : 0;
  if (s.stop == 2) r->status = OM_RES_LIMIT;
  else r->status = r->has_solution ? OM_RES_OPTIMAL : OM_RES_INFEASIBLE;
  if (!r->has_solution) r->objective = 0;
  free(s.dvar); free(s.dkind); free(s.dval); free(s.lb); free(s.ub);
  if (trace_n) *trace_n = s.trace_n;
  return rc;
}

int om_solve(const om_model* m, const om_solve_opts* o, om_solve_result* r, i64* witness) {
  return om_solve_traced(m, o, r, witness, NULL, 0, NULL);
}

/* Batch driver: propagate n stores (row-major [n][n_vars]) one after another
 * in forward order.  status[i] / sweeps[i] per store. */
void om_propagate_batch(const om_model* m, int64_t n, i64* lb, i64* ub, int32_t* status,
                        int64_t* sweeps) {
  for (int64_t i = 0; i < n; ++i) {
    int64_t sw = 0;
    status[i] = om_propagate(m, lb + i * m->n_vars, ub + i * m->n_vars, OM_FORWARD, 0,
                             INT64_MAX, &sw);
    if (sweeps) sweeps[i] = sw;
  }
}
