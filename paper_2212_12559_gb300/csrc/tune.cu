// Launch-shape autotuner (see tune.cuh).
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <sstream>

#include "tune.cuh"

namespace smg {
namespace {

struct Entry {
  int id = 0;
  std::string name;
  std::vector<std::pair<std::string, double>> times;   // name, ms per launch
};

std::mutex g_mu;
std::map<std::string, Entry> g_table;
int g_mode = 1;

}  // namespace

void tune_set_mode(int mode) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_mode = mode ? 1 : 0;
}

int tune_mode() {
  std::lock_guard<std::mutex> lock(g_mu);
  return g_mode;
}

int tune_fastest(const std::vector<double>& ms) {
  int best = -1;
  for (size_t i = 0; i < ms.size(); ++i)
    if (std::isfinite(ms[i]) && (best < 0 || ms[i] < ms[best])) best = (int)i;
  return best;
}

int tune_pick(const std::string& key, const std::vector<TuneCandidate>& cands, cudaStream_t st,
              const std::function<void(int)>& run, int nrep) {
  SMG_REQUIRE(!cands.empty(), "tune_pick: no candidate for " + key);
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_table.find(key);
    if (it != g_table.end()) {
      for (const auto& c : cands)
        if (c.id == it->second.id) return c.id;
      // a loaded entry naming a candidate this shape does not offer: retune
    }
    if (g_mode == 0 || cands.size() == 1) return cands[0].id;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  SMG_CUDA_OK(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return cands[0].id;
  cudaEvent_t e0, e1;
  SMG_CUDA_OK(cudaEventCreate(&e0));
  SMG_CUDA_OK(cudaEventCreate(&e1));
  std::vector<double> ms(cands.size(), NAN);
  for (size_t i = 0; i < cands.size(); ++i) {
    run(cands[i].id);                       // warm-up (and first-launch set-up)
    SMG_CUDA_OK(cudaEventRecord(e0, st));
    for (int r = 0; r < nrep; ++r) run(cands[i].id);
    SMG_CUDA_OK(cudaEventRecord(e1, st));
    SMG_CUDA_OK(cudaEventSynchronize(e1));
    float t = 0.f;
    SMG_CUDA_OK(cudaEventElapsedTime(&t, e0, e1));
    ms[i] = (double)t / nrep;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int b = tune_fastest(ms);
  SMG_REQUIRE(b >= 0, "tune_pick: no candidate could be timed for " + key);
  Entry e;
  e.id = cands[b].id;
  e.name = cands[b].name;
  for (size_t i = 0; i < cands.size(); ++i) e.times.push_back({cands[i].name, ms[i]});
  std::lock_guard<std::mutex> lock(g_mu);
  g_table[key] = e;
  return e.id;
}

std::string tune_table_text() {
  std::lock_guard<std::mutex> lock(g_mu);
  std::ostringstream o;
  for (const auto& kv : g_table) {
    o << kv.first << '\t' << kv.second.id << '\t' << kv.second.name;
    for (const auto& t : kv.second.times) {
      char buf[64];
      std::snprintf(buf, sizeof(buf), "%.6g", t.second);
      o << '\t' << t.first << '=' << buf;
    }
    o << '\n';
  }
  return o.str();
}

int tune_table_load(const std::string& text) {
  std::map<std::string, Entry> add;
  std::istringstream in(text);
  std::string line;
  while (std::getline(in, line)) {
    if (line.empty() || line[0] == '#') continue;
    std::istringstream ls(line);
    std::string key, ids, name;
    if (!std::getline(ls, key, '\t') || !std::getline(ls, ids, '\t') || key.empty()) return -1;
    std::getline(ls, name, '\t');
    char* end = nullptr;
    const long id = std::strtol(ids.c_str(), &end, 10);
    if (end == ids.c_str() || *end != '\0' || id < 0 || id > 1000000) return -1;
    Entry e;
    e.id = (int)id;
    e.name = name;
    add[key] = e;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto& kv : add) g_table[kv.first] = kv.second;
  return (int)add.size();
}

void tune_table_clear() {
  std::lock_guard<std::mutex> lock(g_mu);
  g_table.clear();
}

}  // namespace smg
