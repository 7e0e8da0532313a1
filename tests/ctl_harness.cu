// Host-side driver of the solver's outer-loop functions (ctl_plan, ctl_params, ctl_mid,
// ctl_collect), built and run by tests/test_cycle_ctl_cpu.py without a GPU.  Each scenario
// feeds the functions a sequence of inner-loop outcomes and outer residuals and prints the
// decisions as key=value lines for the test to check against Algorithm 1's reading.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "../paper_1904_08616_gb300/csrc/solver_impl.cuh"

using lq::CycleCtl;
using lq::SolverState;
using namespace lq::solver_detail;

static void init(CycleCtl& c, int nb, double eta_norm, double s0, double tol, double delta, int max_cycles,
                 int max_iter, int per_cycle) {
    memset(&c, 0, sizeof(c));
    c.nb = nb;
    c.delta = delta;
    c.max_cycles = max_cycles;
    c.max_iter = max_iter;
    c.per_cycle = per_cycle;
    for (int j = 0; j < nb; ++j) {
        c.eta_norm[j] = eta_norm;
        c.first[j] = 1;
        c.target[j] = tol * eta_norm;
        c.s[j] = s0;
        c.best[j] = s0;
    }
}

// one cycle for right-hand side 0: iters inner iterations ending at rho (stop code stop),
// then the outer residual s_new
static void cycle(CycleCtl& c, int iters, double rho, int stop, double s_new) {
    SolverState st;
    memset(&st, 0, sizeof(st));
    for (int j = 0; j < c.nb; ++j) {
        st.iter[j] = iters;
        st.rho[j] = rho;
        st.stop[j] = stop;
        st.red[2][j] = s_new * s_new;
    }
    ctl_mid(c, st);
    ctl_collect(c, st);
}

static void show(const char* tag, const CycleCtl& c) {
    printf("%s done=%d status=%d first=%d stagnant=%d total=%d cycles=%d l=%d k_max=%d act=%d cont=%d "
           "is=%.17g stop_rho=%.17g b0=%.17g s=%.17g best=%.17g xact=%d xs=%.17g\n",
           tag, c.done[0], c.status[0], c.first[0], c.stagnant[0], c.total[0], c.cycles[0], c.l, c.k_max, c.act[0],
           c.cont[0], c.is[0], c.stop_rho[0], c.b0[0], c.s[0], c.best[0], c.xact[0], c.xs[0]);
}

int main() {
    CycleCtl c;
    // converging: s drops by 1e-2 per cycle with the recurrence predicting it (rho_k = 1e-4)
    init(c, 1, 2.0, 2.0, 1e-10, 1e-2, 1000, 100000, 1000);
    printf("plan0 %d\n", (int)ctl_plan(c));
    ctl_params(c);
    show("conv0", c);
    double s = 2.0;
    for (int k = 1; k <= 6; ++k) {
        s *= 1e-2;
        cycle(c, 30, 1e-4, 1, s);
        const bool more = ctl_plan(c);
        ctl_params(c);
        char tag[16];
        snprintf(tag, sizeof tag, "conv%d", k);
        printf("plan%d %d\n", k, (int)more);
        show(tag, c);
    }
    // drift: the true residual is 10x what the recurrence predicted -> restart afresh
    init(c, 1, 1.0, 1.0, 1e-10, 1e-2, 1000, 100000, 1000);
    ctl_plan(c);
    ctl_params(c);
    cycle(c, 20, 1e-4, 1, 0.1);
    ctl_plan(c);
    ctl_params(c);
    show("drift", c);
    // stagnation: s never improves on its best by 0.1%
    init(c, 1, 1.0, 1e-3, 1e-10, 1e-2, 1000, 100000, 1000);
    ctl_plan(c);
    ctl_params(c);
    for (int k = 1; k <= 6; ++k) {
        cycle(c, 10, 1e-4, 1, 1e-3);
        printf("stag%d %d\n", k, (int)ctl_plan(c));
        ctl_params(c);
    }
    show("stag", c);
    // caps: max_cycles 2, and a total iteration cap that shrinks k_max
    init(c, 1, 1.0, 1.0, 1e-10, 1e-2, 2, 100000, 1000);
    ctl_plan(c);
    ctl_params(c);
    cycle(c, 10, 1e-4, 1, 1e-2);
    ctl_plan(c);
    ctl_params(c);
    cycle(c, 10, 1e-4, 1, 1e-4);
    printf("plan_maxcyc %d\n", (int)ctl_plan(c));
    show("maxcyc", c);
    init(c, 1, 1.0, 1.0, 1e-10, 1e-2, 1000, 50, 1000);
    ctl_plan(c);
    show("iters0", c);
    cycle(c, 45, 1e-4, 1, 1e-2);
    ctl_plan(c);
    show("iters1", c);
    cycle(c, 5, 1e-4, 1, 1e-4);
    printf("plan_iters2 %d\n", (int)ctl_plan(c));
    show("iters2", c);
    // breakdown and non-finite stops of the inner loop
    init(c, 1, 1.0, 1.0, 1e-10, 1e-2, 1000, 100000, 1000);
    ctl_plan(c);
    ctl_params(c);
    cycle(c, 7, 1e-4, 2, 0.5);
    printf("plan_brk %d\n", (int)ctl_plan(c));
    show("brk", c);
    init(c, 1, 1.0, 1.0, 1e-10, 1e-2, 1000, 100000, 1000);
    ctl_plan(c);
    ctl_params(c);
    cycle(c, 7, 1e-4, 1, NAN);
    printf("plan_nan %d\n", (int)ctl_plan(c));
    show("nan", c);
    return 0;
}
