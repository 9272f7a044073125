// otgs_solver.cuh -- device L-BFGS state and host driver.
#pragma once

#include "otgs_handle.cuh"

namespace otgs {

constexpr int MAX_LBFGS_M = 32;
constexpr int SOLVER_THREADS = 256;
constexpr int TRACE_CAP = 1 << 16;  // objective trace entries kept per solve
constexpr int TRIALS_PER_SYNC = 16;  // line-search trials queued between host checks
// line search (same constants as the oracle)
constexpr double LS_C1 = 1e-4;
constexpr double LS_C2 = 0.9;
constexpr double LS_EPS_F = 1e-12;
constexpr int LS_MAX_EVALS = 40;
// pair-independent dot products
enum { DOT_SY = 0, DOT_SS, DOT_YY, DOT_GG, NBASE };
// per stored slot k: s_new.y_k, s_k.y_new, y_new.y_k, G.s_k, G.y_k
enum { PD_SNEW_Y = 0, PD_S_YNEW, PD_YNEW_Y, PD_G_S, PD_G_Y, NPAIR };

struct SolverState {
    int status, done, iter, npairs, head, accepted, refresh, force_accept;
    int ls_evals, have_hi, M, r, screening, maxit;
    int go;  // the current trial runs (set by the trial gate: not done, no refresh pending)
    long long evals;
    double tol, t, lo, Flo, dlo, hi, Fhi, dhi;
    double F, F0, dphi0, ginf, cG, budget_ns;
    unsigned long long t_start;
    unsigned long long t_begin;  // globaltimer when the solve was launched
    double* trace;               // [trace_cap][3]: D, ms since t_begin, evaluations
    int trace_cap;
    int pad_trace;
    double SY[MAX_LBFGS_M * MAX_LBFGS_M];  // SY[i*M + k] = s_i . y_k
    double YY[MAX_LBFGS_M * MAX_LBFGS_M];
    double cy[MAX_LBFGS_M], cs[MAX_LBFGS_M];
};

struct Solver {
    Handle* h = nullptr;
    int N = 0, M = 0, nblk = 0;
    SolverState* state = nullptr;
    SolverState* hstate = nullptr;  // pinned
    double *x = nullptr, *G = nullptr, *d = nullptr, *xt = nullptr, *Gt = nullptr;
    double *Sv = nullptr, *Yv = nullptr;
    double *pbase = nullptr, *ppair = nullptr;  // dot partials
    double* trace = nullptr;                    // objective trace of the last solve
    int trace_len = 0;
    double D = 0.0, ginf = 0.0;
    int iters = 0;
    ~Solver();
    bool init(Handle* h);
    int run(double tol, int maxit);
    bool eval_trial();
    void launch_dots(bool start);
};

}  // namespace otgs
