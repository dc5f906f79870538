// Batched Algorithm 2 over independent instances: one captured CUDA graph per
// batch, replayed by a single cudaGraphLaunch per call, with a two-level
// autotuner (kernel family per instance, then concurrent branch count).
//
// Blocks of one problem are filtered independently (Sec. 4.4); separate
// problems are independent a fortiori, so their launch sequences can run on
// concurrent branches of one graph.  Everything a captured launch reads from
// the host (the per-block scalar images of Algorithm 2 steps 1, 3, 4) lives in
// pinned buffers owned by the batch and rewritten before every replay; the
// coefficients baked into the kernel nodes depend only on (degree, bounds),
// which are part of the graph's signature.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace {

using pawfe::ChebScalars;
using pawfe::Error;

struct InstPlan {
  bool valid = false;
  paw_status st = PAW_OK;
  std::vector<ChebScalars> blocks;   // one per opts.block columns
  std::vector<size_t> hd_off, hf_off;   // offsets into the pinned arenas
};

}  // namespace

struct paw_batch_s {
  std::vector<paw_context *> inst;
  paw_batch_options opts{};
  int device = 0;
  std::vector<cudaStream_t> lanes;
  cudaStream_t origin = nullptr;         // capture origin (the legacy stream cannot be captured)
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t exec = nullptr;
  size_t graph_nodes = 0, kernel_nodes = 0;
  int captures = 0;
  int branches = 1;
  std::vector<double> sig;               // signature of the captured graph
  double *hd = nullptr;                  // pinned scalar images
  float *hf = nullptr;
  size_t hd_cap = 0, hf_cap = 0;
  std::vector<int> branch_of;            // graph branch of each instance (-1: not in the graph)
  std::vector<std::array<double, 2>> tuned_ms;
};

namespace {

void release_graph(paw_batch_s *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->graph_nodes = 0;
}

void check_problem(paw_context *c, const paw_batch_problem &q) {
  PAW_REQUIRE(q.ncols >= 0, PAW_ERR_INVALID_ARG, "ncols < 0");
  if (q.ncols == 0) return;
  PAW_REQUIRE(q.X_in && q.X_out && q.lambda_in, PAW_ERR_INVALID_ARG, "NULL X_in, X_out or lambda_in");
  PAW_REQUIRE(q.ldx >= q.ncols && q.ldo >= q.ncols, PAW_ERR_INVALID_ARG, "leading dimension smaller than ncols");
  PAW_REQUIRE(q.X_in != q.X_out, PAW_ERR_INVALID_ARG, "X_out must not alias X_in");
  PAW_REQUIRE(q.degree >= 1, PAW_ERR_INVALID_ARG, "degree must be >= 1");
  const paw_bounds &bd = q.bounds;
  PAW_REQUIRE(std::isfinite(bd.a0) && std::isfinite(bd.bW) && std::isfinite(bd.bU) && bd.a0 < bd.bW && bd.bW < bd.bU,
              PAW_ERR_INVALID_ARG, "bounds must satisfy a0 < bW < bU");
  for (int j = 0; j < q.ncols; ++j)
    PAW_REQUIRE(std::isfinite(q.lambda_in[j]), PAW_ERR_NONFINITE, "lambda_in has NaN/Inf");
  (void)c;
}

// Scalars of every block of every valid instance into the pinned arenas.
void fill_scalars(paw_batch_s *b, const paw_batch_problem *pr, std::vector<InstPlan> &plan) {
  for (size_t i = 0; i < b->inst.size(); ++i) {
    InstPlan &P = plan[i];
    if (!P.valid) continue;
    const int B = b->inst[i]->opts.block;
    for (size_t k = 0; k < P.blocks.size(); ++k) {
      const int j0 = (int)k * B, nb = std::min(B, pr[i].ncols - j0);
      pawfe::cheb_plan(nb, pr[i].degree, pr[i].bounds, pr[i].lambda_in + j0, P.blocks[k], b->hd + P.hd_off[k],
                       b->hf + P.hf_off[k]);
    }
  }
}

// Enqueue all blocks of instance i on stream s (no host synchronisation).
void issue_instance(paw_batch_s *b, paw_precision prec, const paw_batch_problem &q, const InstPlan &P, size_t i,
                    cudaStream_t s) {
  paw_context *c = b->inst[i];
  const int B = c->opts.block;
  for (size_t k = 0; k < P.blocks.size(); ++k) {
    const int j0 = (int)k * B, nb = std::min(B, q.ncols - j0);
    pawfe::cheb_issue(c, prec, q.X_in + j0, q.ldx, nb, q.bounds, P.blocks[k], b->hd + P.hd_off[k],
                      b->hf + P.hf_off[k], q.X_out + j0, q.ldo, s);
  }
}

// Capture every valid instance into one graph with `branches` concurrent
// branches.  The capture runs on the batch's own origin stream; the graph is
// launched on the caller's stream.
void capture(paw_batch_s *b, paw_precision prec, const paw_batch_problem *pr, const std::vector<InstPlan> &plan,
             int branches) {
  cudaStream_t s = b->origin;
  release_graph(b);
  std::vector<int> prof_on(b->inst.size());
  for (size_t i = 0; i < b->inst.size(); ++i) {   // no event brackets inside the graph
    prof_on[i] = b->inst[i]->prof.on ? 1 : 0;
    b->inst[i]->prof.on = false;
  }
  cudaGraph_t g = nullptr;
  PAW_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  try {
    PAW_CUDA(cudaEventRecord(b->fork, s));
    for (int l = 0; l < branches; ++l) PAW_CUDA(cudaStreamWaitEvent(b->lanes[l], b->fork, 0));
    int next = 0;
    for (size_t i = 0; i < b->inst.size(); ++i) {
      b->branch_of[i] = -1;
      if (!plan[i].valid) continue;
      b->branch_of[i] = next % branches;
      issue_instance(b, prec, pr[i], plan[i], i, b->lanes[next % branches]);
      ++next;
    }
    for (int l = 0; l < branches; ++l) {
      PAW_CUDA(cudaEventRecord(b->join[l], b->lanes[l]));
      PAW_CUDA(cudaStreamWaitEvent(s, b->join[l], 0));
    }
  } catch (...) {
    cudaStreamEndCapture(s, &g);
    if (g) cudaGraphDestroy(g);
    for (size_t i = 0; i < b->inst.size(); ++i) b->inst[i]->prof.on = prof_on[i] != 0;
    throw;
  }
  PAW_CUDA(cudaStreamEndCapture(s, &g));
  for (size_t i = 0; i < b->inst.size(); ++i) b->inst[i]->prof.on = prof_on[i] != 0;
  const cudaError_t e = cudaGraphInstantiate(&b->exec, g, 0);
  size_t n = 0, nk = 0;
  cudaGraphGetNodes(g, nullptr, &n);
  if (n > 0) {
    std::vector<cudaGraphNode_t> nodes(n);
    cudaGraphGetNodes(g, nodes.data(), &n);
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++nk;
    }
  }
  cudaGraphDestroy(g);
  PAW_CUDA(e);
  b->graph_nodes = n;
  b->kernel_nodes = nk;
  b->branches = branches;
  ++b->captures;
}

float time_graph(paw_batch_s *b, cudaStream_t s) {
  cudaEvent_t e0, e1;
  PAW_CUDA(cudaEventCreate(&e0));
  PAW_CUDA(cudaEventCreate(&e1));
  PAW_CUDA(cudaGraphLaunch(b->exec, s));   // warm
  PAW_CUDA(cudaEventRecord(e0, s));
  PAW_CUDA(cudaGraphLaunch(b->exec, s));
  PAW_CUDA(cudaEventRecord(e1, s));
  PAW_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

// Kernel family of instance i: a short filter (degree <= 4) of its first block
// with each family, timed alone; the faster one is kept.
void tune_instance(paw_batch_s *b, paw_precision prec, const paw_batch_problem &q, size_t i, cudaStream_t s) {
  paw_context *c = b->inst[i];
  b->tuned_ms[i] = {0.0, 0.0};
  c->grid_cap = 0;
  if (prec == PAW_FP64 || c->nown_pairs == 0) {   // FP64 form: no tensor-core kernels to choose between
    c->tc_variant = 0;
    return;
  }
  const int nb = std::min(c->opts.block, q.ncols);
  const int m = std::min(q.degree, 4);
  ChebScalars S;
  std::vector<double> hd(pawfe::cheb_nd(nb, m));
  std::vector<float> hf(pawfe::cheb_nf(nb, m));
  pawfe::cheb_plan(nb, m, q.bounds, q.lambda_in, S, hd.data(), hf.data());
  cudaEvent_t e0, e1;
  PAW_CUDA(cudaEventCreate(&e0));
  PAW_CUDA(cudaEventCreate(&e1));
  float best = 0.f;
  int bestv = 0;
  for (int v = 0; v < 2; ++v) {
    c->tc_variant = v;
    pawfe::cheb_issue(c, prec, q.X_in, q.ldx, nb, q.bounds, S, hd.data(), hf.data(), q.X_out, q.ldo, s);   // warm
    PAW_CUDA(cudaEventRecord(e0, s));
    pawfe::cheb_issue(c, prec, q.X_in, q.ldx, nb, q.bounds, S, hd.data(), hf.data(), q.X_out, q.ldo, s);
    PAW_CUDA(cudaEventRecord(e1, s));
    PAW_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    b->tuned_ms[i][v] = ms;
    if (v == 0 || ms < best) {
      best = ms;
      bestv = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->tc_variant = bestv;
}

int sm_count(int dev) {
  int n = 0;
  PAW_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  return n;
}

}  // namespace

extern "C" {

paw_status paw_batch_create(const paw_handle *handles, int count, const paw_batch_options *options,
                            paw_batch *out) {
  using namespace pawfe;
  paw_batch_s *b = nullptr;
  try {
    PAW_REQUIRE(out != nullptr, PAW_ERR_INVALID_ARG, "NULL out");
    *out = nullptr;
    PAW_REQUIRE(handles != nullptr && count >= 1, PAW_ERR_INVALID_ARG, "need count >= 1 handles");
    for (int i = 0; i < count; ++i) {
      PAW_REQUIRE(handles[i] != nullptr, PAW_ERR_INVALID_ARG, "NULL handle in the batch");
      PAW_REQUIRE(!handles[i]->kc, PAW_ERR_UNSUPPORTED, "batches take handles without a Bloch wavevector");
      for (int j = 0; j < i; ++j)
        PAW_REQUIRE(handles[j] != handles[i], PAW_ERR_INVALID_ARG, "a handle appears twice in the batch");
    }
    b = new paw_batch_s();
    b->inst.assign(handles, handles + count);
    if (options) b->opts = *options;
    if (b->opts.streams <= 0) b->opts.streams = 4;
    b->opts.streams = std::min(b->opts.streams, 8);
    PAW_CUDA(cudaGetDevice(&b->device));
    b->lanes.resize(b->opts.streams);
    b->join.resize(b->opts.streams);
    for (int l = 0; l < b->opts.streams; ++l) {
      PAW_CUDA(cudaStreamCreateWithFlags(&b->lanes[l], cudaStreamNonBlocking));
      PAW_CUDA(cudaEventCreateWithFlags(&b->join[l], cudaEventDisableTiming));
    }
    PAW_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    PAW_CUDA(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking));
    b->branch_of.assign(count, -1);
    b->tuned_ms.assign(count, {0.0, 0.0});
    *out = b;
    return PAW_OK;
  } catch (const Error &err) {
    if (b) paw_batch_destroy(b);
    return fail(err.code, err.msg);
  } catch (const std::exception &ex) {
    if (b) paw_batch_destroy(b);
    return fail(PAW_ERR_CUDA, ex.what());
  }
}

paw_status paw_batch_cheb_filter(paw_batch b, paw_precision prec, const paw_batch_problem *problems,
                                 paw_status *status_out, void *stream) {
  using namespace pawfe;
  try {
    PAW_REQUIRE(b != nullptr && problems != nullptr, PAW_ERR_INVALID_ARG, "NULL batch or problems");
    PAW_REQUIRE(prec == PAW_FP64 || prec == PAW_FP32 || prec == PAW_TF32 || prec == PAW_BF16, PAW_ERR_INVALID_ARG,
                "unknown precision");
    auto s = (cudaStream_t)stream;
    const size_t n = b->inst.size();
    std::vector<InstPlan> plan(n);
    // ---- validation and arena layout; the signature of the launch sequence
    std::vector<double> sig{(double)prec};
    size_t nd = 0, nf = 0;
    for (size_t i = 0; i < n; ++i) {
      InstPlan &P = plan[i];
      const paw_batch_problem &q = problems[i];
      try {
        check_problem(b->inst[i], q);
        P.valid = q.ncols > 0;
      } catch (const Error &err) {
        P.valid = false;
        P.st = err.code;
        set_error(err.msg);
      }
      sig.push_back(P.valid ? 1.0 : 0.0);
      if (!P.valid) continue;
      paw_context *c = b->inst[i];
      c->last_stream = s;
      const int B = c->opts.block;
      for (int j0 = 0; j0 < q.ncols; j0 += B) {
        const int nb = std::min(B, q.ncols - j0);
        P.blocks.emplace_back();
        P.hd_off.push_back(nd);
        P.hf_off.push_back(nf);
        nd += cheb_nd(nb, q.degree);
        nf += cheb_nf(nb, q.degree);
      }
      const double v[] = {(double)(uintptr_t)q.X_in, (double)q.ldx, (double)q.ncols, (double)q.degree, q.bounds.a0,
                          q.bounds.bW, q.bounds.bU, (double)(uintptr_t)q.X_out, (double)q.ldo};
      sig.insert(sig.end(), v, v + 9);
    }
    bool rebuild = b->exec == nullptr || sig != b->sig;
    if (nd > b->hd_cap || nf > b->hf_cap) {   // captured copies read the arenas: new arenas, new graph
      PAW_CUDA(cudaStreamSynchronize(s));
      if (b->hd) cudaFreeHost(b->hd);
      if (b->hf) cudaFreeHost(b->hf);
      b->hd = nullptr;
      b->hf = nullptr;
      b->hd_cap = std::max<size_t>(nd, 1);
      b->hf_cap = std::max<size_t>(nf, 1);
      PAW_CUDA(cudaMallocHost(&b->hd, sizeof(double) * b->hd_cap));
      PAW_CUDA(cudaMallocHost(&b->hf, sizeof(float) * b->hf_cap));
      rebuild = true;
    }
    fill_scalars(b, problems, plan);

    bool any = false;
    for (size_t i = 0; i < n; ++i) any = any || plan[i].valid;
    if (any) {
      if (rebuild) {
        PAW_CUDA(cudaStreamSynchronize(s));
        int nvalid = 0;
        for (size_t i = 0; i < n; ++i) {
          if (!plan[i].valid) continue;
          ++nvalid;
          if (b->opts.autotune) tune_instance(b, prec, problems[i], i, s);
          // one uncaptured pass: every workspace and operand image exists before capture
          issue_instance(b, prec, problems[i], plan[i], i, s);
        }
        PAW_CUDA(cudaStreamSynchronize(s));
        const int maxbr = std::max(1, std::min(b->opts.streams, nvalid));
        const int nsm = sm_count(b->device);
        if (b->opts.autotune && maxbr > 1) {
          float best = 0.f;
          int bestbr = 1;
          for (int br = 1; br <= maxbr; br *= 2) {
            for (size_t i = 0; i < n; ++i) b->inst[i]->grid_cap = br > 1 ? (nsm + br - 1) / br : 0;
            capture(b, prec, problems, plan, br);
            const float ms = time_graph(b, s);
            if (br == 1 || ms < best) {
              best = ms;
              bestbr = br;
            }
          }
          for (size_t i = 0; i < n; ++i) b->inst[i]->grid_cap = bestbr > 1 ? (nsm + bestbr - 1) / bestbr : 0;
          capture(b, prec, problems, plan, bestbr);
        } else {
          for (size_t i = 0; i < n; ++i) b->inst[i]->grid_cap = maxbr > 1 ? (nsm + maxbr - 1) / maxbr : 0;
          capture(b, prec, problems, plan, maxbr);
        }
        b->sig = sig;
      }
      PAW_CUDA(cudaGraphLaunch(b->exec, s));
      PAW_CUDA(cudaStreamSynchronize(s));
    }
    paw_status first = PAW_OK;
    for (size_t i = 0; i < n; ++i) {
      paw_status st = plan[i].st;
      if (plan[i].valid && (prec == PAW_TF32 || prec == PAW_BF16)) {
        const int v = read_status(b->inst[i]);
        if (v != 0) st = (v < 0) ? PAW_ERR_CUDA : PAW_ERR_TIMEOUT;
      }
      if (status_out) status_out[i] = st;
      if (first == PAW_OK && st != PAW_OK) first = st;
    }
    if (first != PAW_OK) set_error("paw_batch_cheb_filter: at least one instance failed (see status_out)");
    return first;
  } catch (const Error &err) {
    return fail(err.code, err.msg);
  } catch (const std::exception &ex) {
    return fail(PAW_ERR_CUDA, ex.what());
  }
}

paw_status paw_batch_tuning_get(paw_batch b, int i, paw_batch_tuning *out) {
  using namespace pawfe;
  if (!b || !out || i < 0 || i >= (int)b->inst.size()) return fail(PAW_ERR_INVALID_ARG, "bad batch, index or out");
  paw_context *c = b->inst[i];
  std::memset(out, 0, sizeof(*out));
  out->tc_variant = c->tc_variant;
  out->grid_cap = c->grid_cap;
  out->branches = b->branches;
  out->branch = b->branch_of[i];
  out->graph_nodes = (int32_t)b->graph_nodes;
  out->kernel_nodes = (int32_t)b->kernel_nodes;
  out->captures = b->captures;
  out->tuned_ms[0] = b->tuned_ms[i][0];
  out->tuned_ms[1] = b->tuned_ms[i][1];
  return PAW_OK;
}

paw_status paw_batch_destroy(paw_batch b) {
  if (!b) return PAW_OK;
  release_graph(b);
  for (auto l : b->lanes)
    if (l) cudaStreamDestroy(l);
  for (auto e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->hd) cudaFreeHost(b->hd);
  if (b->hf) cudaFreeHost(b->hf);
  for (auto *c : b->inst) {   // back to the single-instance defaults
    c->tc_variant = 0;
    c->grid_cap = 0;
  }
  delete b;
  return PAW_OK;
}

}  // extern "C"
