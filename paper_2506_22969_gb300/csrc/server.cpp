// Stencil-job server: a request loop over the sparse sweep library (north-of-kernel runtime).
//
// Jobs (a stencil, a grid on the host, a step count) arrive over time.  A dispatcher thread
// admits them in arrival order as execution slots (CUDA streams) and device memory under an
// HBM budget become free, so that work submitted while other jobs are on the GPU joins them
// there: each admitted job copies its grid in (unless it is already on the device), runs its
// sweeps and copies the result out (unless it stays on the device) on its own stream, side by
// side with the others.  Plans are kept per stencil signature and reused by later jobs (a
// plan holds device tables and a workspace, so one plan serves one job at a time).  The
// server's grids and workspaces come from a stream-ordered memory pool of its own whose
// release threshold is the budget, so memory freed by a job stays resident for the next.
// 2D and 3D jobs run the sparse tensor-core path.  Latencies (completion minus arrival) give
// p50/p99.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "sparstencil.h"

namespace spst {
sparstencil_status report_error(sparstencil_status s, const char* msg);
}

namespace {

// ---------------------------------------------------------------------------------------
// Admission policy (host only; also driven by the simulator entry point for tests).
// ---------------------------------------------------------------------------------------
struct Policy {
  size_t budget;
  int slots;
  size_t in_use = 0;
  int busy = 0;
  // FIFO: the head job is admitted when a slot is free and its bytes fit next to the bytes in
  // use; later jobs wait behind it (no overtaking, so no job starves).
  bool can_admit(size_t bytes) const { return busy < slots && in_use + bytes <= budget; }
  void admit(size_t bytes) {
    in_use += bytes;
    busy++;
  }
  void release(size_t bytes) {
    in_use -= bytes;
    busy--;
  }
};

struct Job {
  int64_t id = 0;
  sparstencil_shape shape = SPST_BOX;
  int radius = 1, ndim = 2, fusion = 1;
  std::vector<float> weights;
  std::vector<int64_t> dims;
  sparstencil_dtype dtype = SPST_BF16;
  sparstencil_boundary bc = SPST_PERIODIC;
  int64_t steps = 0;
  const float* in_host = nullptr;
  float* out_host = nullptr;
  const float* in_dev = nullptr;  // caller-owned device grids (resident across jobs)
  float* out_dev = nullptr;
  double arrival = 0, admitted = -1, done = -1;
  size_t bytes = 0;
  int status = SPST_OK;
  // while running
  int slot = -1;
  sparstencil_plan_t plan = nullptr;
  std::string key;
  float *d_in = nullptr, *d_out = nullptr;
  void* d_ws = nullptr;
  size_t ws_bytes = 0;
  cudaEvent_t finished = nullptr;
};

std::string plan_key(const Job& j) {
  std::string k;
  auto put = [&](const void* p, size_t n) { k.append((const char*)p, n); };
  put(&j.shape, sizeof(j.shape));
  put(&j.radius, sizeof(j.radius));
  put(&j.ndim, sizeof(j.ndim));
  put(&j.fusion, sizeof(j.fusion));
  put(&j.dtype, sizeof(j.dtype));
  put(&j.bc, sizeof(j.bc));
  put(j.dims.data(), j.dims.size() * sizeof(int64_t));
  put(j.weights.data(), j.weights.size() * sizeof(float));
  return k;
}

int64_t cells(const Job& j) {
  int64_t n = 1;
  for (auto d : j.dims) n *= d;
  return n;
}

}  // namespace

struct sparstencil_server_s {
  int device = 0;
  Policy policy;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Job>> pending;
  std::vector<std::shared_ptr<Job>> running;
  std::map<int64_t, std::shared_ptr<Job>> finished;
  std::multimap<std::string, sparstencil_plan_t> idle_plans;
  std::vector<cudaStream_t> streams;
  std::vector<char> slot_busy;
  cudaMemPool_t pool = nullptr;  // the server's device allocations (release threshold: the budget)
  int64_t next_id = 1;
  int64_t submitted = 0, completed = 0, failed = 0;
  int64_t point_steps = 0;
  size_t peak_bytes = 0;
  double first_arrival = -1, last_done = 0;
  bool stop = false;
  std::thread worker;

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }

  // Takes the job's plan (an idle one of the same stencil and grid, else a new one: host
  // planning only) and returns the device bytes the job holds while it runs: the grids the
  // server allocates for it (input and output unless the caller's are on the device) plus the
  // plan's workspace.  The planner tables kept on the device by pooled plans are small and
  // not counted.
  size_t take_plan(Job& j, sparstencil_status* st) {
    const size_t grid = (size_t)cells(j) * sizeof(float);
    *st = SPST_OK;
    j.key = plan_key(j);
    auto it = idle_plans.find(j.key);
    if (it != idle_plans.end()) {
      j.plan = it->second;
      idle_plans.erase(it);
    } else {
      *st = sparstencil_plan(j.shape, j.radius, j.weights.data(), j.ndim, j.dims.data(), j.dtype, j.bc, j.fusion,
                             &j.plan);
      if (*st != SPST_OK) return 0;
    }
    j.ws_bytes = sparstencil_workspace_bytes(j.plan);
    return (j.in_dev ? 0 : grid) + (j.out_dev ? 0 : grid) + j.ws_bytes;
  }

  void start_job(const std::shared_ptr<Job>& jp) {
    Job& j = *jp;
    int slot = 0;
    while (slot_busy[slot]) slot++;
    slot_busy[slot] = 1;
    j.slot = slot;
    cudaStream_t s = streams[slot];
    const size_t grid = (size_t)cells(j) * sizeof(float);
    sparstencil_status st = SPST_OK;
    auto alloc = [&](void** p, size_t n) { return cudaMallocFromPoolAsync(p, n, pool, s) == cudaSuccess; };
    float* own_in = nullptr;
    float* own_out = nullptr;
    if ((!j.in_dev && !alloc((void**)&own_in, grid)) || (!j.out_dev && !alloc((void**)&own_out, grid)))
      st = SPST_ERR_NOMEM;
    j.d_in = j.in_dev ? const_cast<float*>(j.in_dev) : own_in;
    j.d_out = j.out_dev ? j.out_dev : own_out;
    if (st == SPST_OK && own_in && cudaMemcpyAsync(own_in, j.in_host, grid, cudaMemcpyHostToDevice, s) != cudaSuccess)
      st = SPST_ERR_CUDA;
    if (st == SPST_OK) {
      // the workspace is the job's, stream-ordered like its grids, and leaves with it
      if (!alloc(&j.d_ws, j.ws_bytes)) st = SPST_ERR_NOMEM;
      if (st == SPST_OK) st = sparstencil_bind_workspace(j.plan, j.d_ws, j.ws_bytes, s);
      if (st == SPST_OK) st = sparstencil_run(j.plan, j.d_in, j.d_out, j.steps, s);
    }
    if (st == SPST_OK && own_out &&
        cudaMemcpyAsync(j.out_host, own_out, grid, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = SPST_ERR_CUDA;
    if (own_in) cudaFreeAsync(own_in, s);
    if (own_out) cudaFreeAsync(own_out, s);
    if (j.d_ws) cudaFreeAsync(j.d_ws, s);
    if (cudaEventCreateWithFlags(&j.finished, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(j.finished, s) != cudaSuccess)
      st = st == SPST_OK ? SPST_ERR_CUDA : st;
    j.status = st;
  }

  void finish_job(const std::shared_ptr<Job>& jp) {
    Job& j = *jp;
    j.done = now();
    if (j.finished) cudaEventDestroy(j.finished);
    j.finished = nullptr;
    slot_busy[j.slot] = 0;
    policy.release(j.bytes);
    if (j.plan) idle_plans.emplace(j.key, j.plan);
    j.plan = nullptr;
    if (j.status == SPST_OK) {
      completed++;
      point_steps += cells(j) * j.steps;
      last_done = std::max(last_done, j.done);
    } else {
      failed++;
    }
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      // completions
      for (size_t i = 0; i < running.size();) {
        auto& jp = running[i];
        const cudaError_t q = jp->finished ? cudaEventQuery(jp->finished) : cudaSuccess;
        if (q == cudaErrorNotReady) {
          i++;
          continue;
        }
        if (q != cudaSuccess && jp->status == SPST_OK) jp->status = SPST_ERR_CUDA;
        finish_job(jp);
        finished[jp->id] = jp;
        running.erase(running.begin() + (long)i);
        cv_done.notify_all();
      }
      // admissions (FIFO)
      while (!pending.empty()) {
        auto jp = pending.front();
        if (jp->bytes > policy.budget) {  // can never fit: fail it
          jp->status = SPST_ERR_NOMEM;
          jp->done = now();
          if (jp->plan) idle_plans.emplace(jp->key, jp->plan);
          jp->plan = nullptr;
          failed++;
          finished[jp->id] = jp;
          pending.pop_front();
          cv_done.notify_all();
          continue;
        }
        if (!policy.can_admit(jp->bytes)) break;
        pending.pop_front();
        policy.admit(jp->bytes);
        peak_bytes = std::max(peak_bytes, policy.in_use);
        jp->admitted = now();
        start_job(jp);
        running.push_back(jp);
      }
      if (stop && pending.empty() && running.empty()) break;
      if (running.empty())
        cv_work.wait(lk, [&] { return stop || !pending.empty(); });
      else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        lk.lock();
      }
    }
  }
};

extern "C" {

sparstencil_status sparstencil_server_create(size_t hbm_budget_bytes, int slots, sparstencil_server_t* out) {
  if (!out) return spst::report_error(SPST_ERR_INVALID, "out is null");
  *out = nullptr;
  if (slots < 1 || slots > 64) return spst::report_error(SPST_ERR_INVALID, "slots must be in 1..64");
  if (hbm_budget_bytes == 0) return spst::report_error(SPST_ERR_INVALID, "budget must be positive");
  std::unique_ptr<sparstencil_server_s> s(new (std::nothrow) sparstencil_server_s());
  if (!s) return spst::report_error(SPST_ERR_NOMEM, "host allocation failed");
  if (cudaGetDevice(&s->device) != cudaSuccess) return spst::report_error(SPST_ERR_CUDA, "cudaGetDevice failed");
  s->policy.budget = hbm_budget_bytes;
  s->policy.slots = slots;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = s->device;
  if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess)
    return spst::report_error(SPST_ERR_CUDA, "memory pool creation failed");
  uint64_t keep = hbm_budget_bytes;  // memory freed by a job stays in the pool up to the budget
  if (cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
    cudaMemPoolDestroy(s->pool);
    return spst::report_error(SPST_ERR_CUDA, "memory pool threshold failed");
  }
  s->streams.assign(slots, nullptr);
  s->slot_busy.assign(slots, 0);
  for (auto& st : s->streams)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : s->streams)
        if (x) cudaStreamDestroy(x);
      cudaMemPoolDestroy(s->pool);
      return spst::report_error(SPST_ERR_CUDA, "stream creation failed");
    }
  sparstencil_server_s* raw = s.get();
  raw->worker = std::thread([raw] { raw->loop(); });
  *out = s.release();
  return SPST_OK;
}

double sparstencil_server_clock(sparstencil_server_t server) { return server ? server->now() : 0.0; }

sparstencil_status sparstencil_server_submit(sparstencil_server_t server, const sparstencil_job* job,
                                             int64_t* job_id) {
  if (!server || !job || !job->weights || !job->dims)
    return spst::report_error(SPST_ERR_INVALID, "null server, job or job pointer");
  if (!job->in_host == !job->in_device || !job->out_host == !job->out_device)
    return spst::report_error(SPST_ERR_INVALID, "give exactly one of in_host / in_device and of out_host / out_device");
  if (job->in_device && (const void*)job->in_device == (const void*)job->out_device)
    return spst::report_error(SPST_ERR_INVALID, "in_device and out_device must not alias");
  if (job->ndim != 2 && job->ndim != 3) return spst::report_error(SPST_ERR_UNSUPPORTED, "ndim must be 2 or 3");
  if (job->timesteps < 0 || job->radius < 1) return spst::report_error(SPST_ERR_INVALID, "bad steps or radius");
  auto jp = std::make_shared<Job>();
  Job& j = *jp;
  j.shape = job->shape;
  j.radius = job->radius;
  j.ndim = job->ndim;
  j.fusion = job->fusion_depth;
  const int side = 2 * job->radius + 1;
  j.weights.assign(job->weights, job->weights + (job->ndim == 3 ? side * side * side : side * side));
  j.dims.assign(job->dims, job->dims + job->ndim);
  for (auto d : j.dims)
    if (d <= 0) return spst::report_error(SPST_ERR_INVALID, "grid extents must be positive");
  j.dtype = job->dtype;
  j.bc = job->bc;
  j.steps = job->timesteps;
  j.in_host = job->in_host;
  j.out_host = job->out_host;
  j.in_dev = job->in_device;
  j.out_dev = job->out_device;
  std::lock_guard<std::mutex> lk(server->mu);
  if (server->stop) return spst::report_error(SPST_ERR_INVALID, "server is shutting down");
  sparstencil_status st = SPST_OK;
  j.bytes = server->take_plan(j, &st);
  if (st != SPST_OK) return st;
  j.arrival = job->arrival_s >= 0 ? job->arrival_s : server->now();
  j.id = server->next_id++;
  if (server->first_arrival < 0 || j.arrival < server->first_arrival) server->first_arrival = j.arrival;
  server->submitted++;
  server->pending.push_back(jp);
  if (job_id) *job_id = j.id;
  server->cv_work.notify_one();
  return SPST_OK;
}

sparstencil_status sparstencil_server_wait(sparstencil_server_t server, int64_t job_id, double timeout_s,
                                           sparstencil_job_result* res) {
  if (!server) return spst::report_error(SPST_ERR_INVALID, "server is null");
  std::unique_lock<std::mutex> lk(server->mu);
  const bool ok = server->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                           [&] { return server->finished.count(job_id) > 0; });
  if (!ok) return spst::report_error(SPST_ERR_TIMEOUT, "job not finished within the timeout");
  const Job& j = *server->finished[job_id];
  if (res) {
    res->job_id = j.id;
    res->status = j.status;
    res->arrival_s = j.arrival;
    res->admit_s = j.admitted;
    res->done_s = j.done;
    res->device_bytes = j.bytes;
  }
  return SPST_OK;
}

sparstencil_status sparstencil_server_drain(sparstencil_server_t server, double timeout_s) {
  if (!server) return spst::report_error(SPST_ERR_INVALID, "server is null");
  std::unique_lock<std::mutex> lk(server->mu);
  const bool ok = server->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
    return server->pending.empty() && server->running.empty();
  });
  return ok ? SPST_OK : spst::report_error(SPST_ERR_TIMEOUT, "jobs still running after the timeout");
}

sparstencil_status sparstencil_server_stats(sparstencil_server_t server, sparstencil_server_summary* out) {
  if (!server || !out) return spst::report_error(SPST_ERR_INVALID, "null server or stats");
  std::lock_guard<std::mutex> lk(server->mu);
  std::memset(out, 0, sizeof(*out));
  std::vector<double> lat;
  for (auto& kv : server->finished)
    if (kv.second->status == SPST_OK) lat.push_back(kv.second->done - kv.second->arrival);
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double q) {
    if (lat.empty()) return 0.0;
    const size_t i = (size_t)std::min<double>((double)lat.size() - 1, q * (double)(lat.size() - 1) + 0.5);
    return lat[i];
  };
  out->submitted = server->submitted;
  out->completed = server->completed;
  out->failed = server->failed;
  out->p50_s = pct(0.50);
  out->p99_s = pct(0.99);
  double sum = 0;
  for (double v : lat) sum += v;
  out->mean_s = lat.empty() ? 0 : sum / (double)lat.size();
  out->max_s = lat.empty() ? 0 : lat.back();
  out->peak_bytes = server->peak_bytes;
  const double span = server->last_done - server->first_arrival;
  out->gstencil_per_s = span > 0 ? (double)server->point_steps / span / 1e9 : 0;
  uint64_t cur = 0, high = 0;
  cudaMemPoolGetAttribute(server->pool, cudaMemPoolAttrReservedMemCurrent, &cur);
  cudaMemPoolGetAttribute(server->pool, cudaMemPoolAttrReservedMemHigh, &high);
  out->pool_reserved_bytes = (size_t)cur;
  out->pool_high_bytes = (size_t)high;
  return SPST_OK;
}

sparstencil_status sparstencil_server_destroy(sparstencil_server_t server) {
  if (!server) return spst::report_error(SPST_ERR_INVALID, "server is null");
  {
    std::lock_guard<std::mutex> lk(server->mu);
    server->stop = true;
  }
  server->cv_work.notify_all();
  if (server->worker.joinable()) server->worker.join();
  for (auto s : server->streams) cudaStreamSynchronize(s);
  for (auto& kv : server->idle_plans) sparstencil_plan_destroy(kv.second);
  for (auto s : server->streams) cudaStreamDestroy(s);
  cudaMemPoolDestroy(server->pool);
  delete server;
  return SPST_OK;
}

// Replays the admission policy on the host for jobs with given arrival times, durations and
// device bytes (no GPU work): admit_s[i] and done_s[i] receive each job's admission and
// completion times, -1 for a job that can never fit the budget.  A job admitted at time a
// completes at a + duration_s[i].
sparstencil_status sparstencil_server_simulate(size_t hbm_budget_bytes, int slots, int n, const double* arrival_s,
                                               const double* duration_s, const size_t* bytes, double* admit_s,
                                               double* done_s) {
  if (n < 0 || slots < 1 || (n > 0 && (!arrival_s || !duration_s || !bytes || !admit_s || !done_s)))
    return spst::report_error(SPST_ERR_INVALID, "bad simulation arguments");
  Policy pol;
  pol.budget = hbm_budget_bytes;
  pol.slots = slots;
  std::vector<int> order(n);
  for (int i = 0; i < n; i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return arrival_s[a] < arrival_s[b]; });
  std::vector<std::pair<double, int>> run;  // (done time, job)
  double t = 0;
  size_t head = 0;
  while (head < order.size() || !run.empty()) {
    // the next event: an arrival of the head job or a completion
    const int h = head < order.size() ? order[head] : -1;
    if (h >= 0 && bytes[h] > pol.budget) {
      admit_s[h] = done_s[h] = -1;
      head++;
      continue;
    }
    if (h >= 0 && arrival_s[h] <= t && pol.can_admit(bytes[h])) {
      pol.admit(bytes[h]);
      admit_s[h] = t;
      done_s[h] = t + duration_s[h];
      run.push_back({done_s[h], h});
      head++;
      continue;
    }
    double next = 1e300;
    if (h >= 0 && arrival_s[h] > t) next = arrival_s[h];
    for (auto& r : run) next = std::min(next, r.first);
    if (next == 1e300) break;
    t = std::max(t, next);
    for (size_t i = 0; i < run.size();) {
      if (run[i].first <= t) {
        pol.release(bytes[run[i].second]);
        run.erase(run.begin() + (long)i);
      } else {
        i++;
      }
    }
  }
  return SPST_OK;
}

}  // extern "C"
