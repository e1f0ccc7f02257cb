// solve.cuh -- internal interface of the solve phase (V-cycle, Krylov drivers).
#pragma once

#include "amg_common.cuh"

struct amg_batch_ws;  // batched-solve work space (batched.cu)

namespace amg {

// Per-kernel tracing: when on, every solve-phase launch is bracketed by CUDA
// events on the launching stream; durations and algorithmic bytes accumulate
// per (kernel, level).  Launches are counted whether or not tracing is on.
struct Profiler {
    struct Rec {
        char name[32];
        int level;
        long long launches;
        double ms;
        double bytes;
    };
    struct Pending {
        int rec;
        cudaEvent_t a, b;
    };
    bool on = false;
    long long launches = 0;
    std::vector<Rec> recs;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    int find(const char *name, int level);
    cudaEvent_t event();
    int collect();  // call after the stream has been synchronised
    void reset();
    void destroy();
};

struct ProfScope {
    Profiler *p;
    cudaStream_t s;
    int rec = -1;
    cudaEvent_t a = nullptr;
    ProfScope(Profiler *p_, cudaStream_t s_, const char *name, int level, double bytes);
    ~ProfScope();
};

// Krylov state shared by all hierarchies of a handle (vectors of length n).
struct Workspace {
    int n = 0;
    double *b = nullptr, *x = nullptr;                     // right-hand side / solution (handle-owned)
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    double *rh = nullptr, *v = nullptr, *ph = nullptr, *s = nullptr, *sh = nullptr, *t = nullptr;
    double *aux = nullptr;                                 // adjoint: forward solution x
    float *r32 = nullptr;                                  // mixed PCG: FP32 copy of r (the V-cycle's input)
    DF *p2 = nullptr;                                      // mixed PCG: p split into FP32 pairs (double-FP32 product)
    DevScalars *scal = nullptr;                            // device
    DevScalars *scal_h = nullptr;                          // pinned host mirror
    double *part = nullptr;                                // per-block partial sums (3 x part_cap)
    unsigned *counter = nullptr;                           // last-block ticket
    unsigned *gbar = nullptr;                              // grid barrier of the fused coarse levels
    int part_cap = 0;
    DevArena arena;
    Profiler prof;
};

int workspace_init(Workspace &W, int n);

// Refines the hierarchy's streaming plans by timed trial (runs whole cycles
// on the workspace's vectors to choose between plan families).
int autotune_plans(Hierarchy *h, Workspace &W, cudaStream_t s);
void workspace_free(Workspace &W);

struct SolveResult {
    int status = AMG_OK, iters = 0, restarts = 0;
    double rel_res_true = 0.0, rel_res_rec = 0.0;
};

// Solves A x = W.b (A = h's finest operator) into W.x with h's configuration.
int krylov_solve(Hierarchy *h, Workspace &W, cudaStream_t s, SolveResult *res);

// Arms the one-shot test control of the bounded waits (AMG_TEST_WITHHOLD_*; 0 disarms).
int test_arm_wait_timeout(Workspace &W, int kind, cudaStream_t s);

// Average duration (us) of the finest Krylov product over reps back-to-back launches.
int time_product(Hierarchy *h, Workspace &W, int reps, cudaStream_t s, double *us);

// z = M^-1 r with one V-cycle of h (r, z: device vectors of length n).
int vcycle_apply(Hierarchy *h, Workspace &W, const double *r, double *z, cudaStream_t s);

// dA[k] = -lambda[row(k)] * x[col(k)] on h's finest pattern.
int grad_values(Hierarchy *h, Workspace &W, const double *lambda, const double *x, double *dA, cudaStream_t s);

// Block-diagonal batches (h->nsys > 0): work space for up to 8 right-hand
// sides per system, and the solve of every (system, right-hand side) pair.
// B: [n][nrhs] (host or device), X likewise; iters / rel_res: [nsys][nrhs]
// (host or device, may be null); res: worst status, largest iteration count
// and largest relative residuals over the pairs.
int batch_create(Hierarchy *h, amg_batch_ws **out);
void batch_destroy(amg_batch_ws *W);
int batch_solve(Hierarchy *h, amg_batch_ws *W, Profiler &prof, int nrhs, const double *B, double *X, int *iters,
                double *rel_res, cudaStream_t s, SolveResult *res);

}  // namespace amg
