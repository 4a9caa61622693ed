// batch.cu -- many independent solves at once (a batch of mapped problems): a
// host-side scheduler drives every context's refinement loop as a small
// state machine.  Each context works on its own stream; each refinement step
// is enqueued without blocking (iteration graphs, then the FP64 residual and
// an asynchronous copy of the device scalars to pinned host memory, then an
// event), and the scheduler polls the events, so small problems overlap with
// each other and with large ones instead of queueing behind host round trips.
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"

namespace bmg {

bmg_status capture_iteration(Ctx& c, int parity);
bmg_status run_iteration(Ctx& c, int parity);
bmg_status stage_in_async(Ctx& c, const double* src, double* dst);
bmg_status stage_out_async(Ctx& c, const double* src, double* dst);
void fill_complexity_info(const Ctx& c, bmg_info* info);

namespace {

struct Job {
    Ctx* c = nullptr;
    int rhs = 0, nrhs = 0;
    const double* const* b = nullptr;
    double* const* x = nullptr;
    bmg_info* info = nullptr;
    cudaEvent_t ev = nullptr;
    int phase = 0;           // 0: idle, 1: waiting for the initial residual, 2: waiting for a refinement
    int it = 0, refinements = 0, m = 0;
    double bb = 0, rr = 0, rr0 = 0, rho = 0.3;
    bool done = false;
    bmg_status status = BMG_OK;
};

bmg_status post_state_copy(Job& j) {
    Ctx& c = *j.c;
    BMG_CUDA(cudaMemcpyAsync(c.st_host, c.st, sizeof(KState), cudaMemcpyDeviceToHost, c.stream));
    BMG_CUDA(cudaEventRecord(j.ev, c.stream));
    return BMG_OK;
}

bmg_status start_rhs(Job& j) {
    Ctx& c = *j.c;
    BMG_TRY(stage_in_async(c, j.b[j.rhs], c.bvec));
    BMG_TRY(stage_in_async(c, j.x[j.rhs], c.x));
    memset(c.st_host, 0, sizeof(KState));
    BMG_CUDA(cudaMemcpyAsync(c.st, c.st_host, sizeof(KState), cudaMemcpyHostToDevice, c.stream));
    BMG_TRY(k_dot(c, c.bvec, c.bvec, &c.st->bb));
    BMG_TRY(k_residual_to32(c));
    BMG_TRY(post_state_copy(j));
    j.phase = 1;
    j.it = j.refinements = 0;
    j.rho = 0.3;
    return BMG_OK;
}

bmg_status finish_rhs(Job& j, double tol) {
    Ctx& c = *j.c;
    BMG_TRY(stage_out_async(c, c.x, j.x[j.rhs]));
    if (j.info) {
        bmg_info& in = j.info[j.rhs];
        in.iterations = j.it;
        in.refinements = j.refinements;
        in.relres = j.bb > 0 ? sqrt(j.rr / j.bb) : 0.0;
        in.true_relres = in.relres;
        in.rho = (j.it > 0 && j.rr0 > 0 && j.rr > 0) ? pow(j.rr / j.rr0, 0.5 / j.it) : 0.0;
        fill_complexity_info(c, &in);
        in.status = j.status;
    }
    (void)tol;
    j.rhs++;
    if (j.rhs < j.nrhs && j.status == BMG_OK) return start_rhs(j);
    j.done = true;
    j.phase = 0;
    return BMG_OK;
}

// Called when the job's event has completed: decide and enqueue the next step.
bmg_status advance(Job& j, double tol, int maxit) {
    Ctx& c = *j.c;
    const KState& h = *c.st_host;
    if (h.err) {
        j.status = (bmg_status)h.err;
        return finish_rhs(j, tol);
    }
    if (j.phase == 1) {
        j.bb = h.bb;
        j.rr = j.rr0 = h.rr;
        if (j.bb == 0.0) {
            BMG_CUDA(cudaMemsetAsync(c.x, 0, sizeof(double) * c.lev[0].plane, c.stream));
            j.rr = 0.0;
            return finish_rhs(j, tol);
        }
    } else {
        const double red = sqrt(h.rr / j.rr);
        if (red > 0 && red < 1) {
            const double r1 = pow(red, 1.0 / j.m);
            if (r1 > 0.02 && r1 < 0.999) j.rho = r1;
        }
        j.rr = h.rr;
        j.refinements++;
    }
    const double lim = tol * tol * j.bb;
    if (j.rr <= lim) return finish_rhs(j, tol);
    if (j.it >= maxit) {
        j.status = BMG_ERR_NOT_CONVERGED;
        return finish_rhs(j, tol);
    }
    double want = sqrt(lim / j.rr);
    if (want < 1e-6) want = 1e-6;
    int m = (int)ceil(log(want) / log(j.rho)) + 1;
    if (m < 2) m = 2;
    if (m > kMaxInner) m = kMaxInner;
    if (m > maxit - j.it) m = maxit - j.it;
    for (int k = 0; k < m; k++) BMG_TRY(run_iteration(c, (j.it + k) & 1));
    j.it += m;
    j.m = m;
    BMG_TRY(k_residual_to32(c));
    BMG_TRY(post_state_copy(j));
    j.phase = 2;
    return BMG_OK;
}

}  // namespace

bmg_status solve_many(Ctx** cs, int count, int nrhs, const double* const* b, double* const* x, double tol,
                      int maxit, bmg_info* infos) {
    std::vector<Job> jobs(count);
    bmg_status st = BMG_OK;
    for (int p = 0; p < count && st == BMG_OK; p++) {
        Job& j = jobs[p];
        j.c = cs[p];
        j.nrhs = nrhs;
        j.b = b + (long long)p * nrhs;
        j.x = x + (long long)p * nrhs;
        j.info = infos ? infos + (long long)p * nrhs : nullptr;
        if (cudaEventCreateWithFlags(&j.ev, cudaEventDisableTiming) != cudaSuccess) st = BMG_ERR_DEVICE;
    }
    // capture the iteration graphs before any launch, so that no capture
    // happens inside the scheduling loop
    for (int p = 0; p < count && st == BMG_OK; p++)
        for (int par = 0; par < 2 && st == BMG_OK; par++) st = capture_iteration(*jobs[p].c, par);
    for (int p = 0; p < count && st == BMG_OK; p++) st = start_rhs(jobs[p]);
    int left = count;
    while (st == BMG_OK && left > 0) {
        for (int p = 0; p < count && st == BMG_OK; p++) {
            Job& j = jobs[p];
            if (j.done) continue;
            const cudaError_t q = cudaEventQuery(j.ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                st = BMG_ERR_DEVICE;
                break;
            }
            st = advance(j, tol, maxit);
            if (j.done) left--;
        }
    }
    for (int p = 0; p < count; p++) {
        if (jobs[p].c) cudaStreamSynchronize(jobs[p].c->stream);
        if (jobs[p].ev) cudaEventDestroy(jobs[p].ev);
    }
    if (st != BMG_OK) return st;
    for (int p = 0; p < count; p++)
        if (jobs[p].status != BMG_OK) return jobs[p].status;
    return BMG_OK;
}

}  // namespace bmg
