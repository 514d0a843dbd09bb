// Launch-shape autotuner.
//
// The multi-RHS kernels take their CTA size from here.  The first launch of a
// (kernel, lattice, nrhs, precision, GPU) combination times every candidate
// with CUDA events on the caller's stream (a few launches each, on the real
// operands) and keeps the fastest; later launches look the choice up.  The
// table lives for the process and, when MGCLOVER_TUNE_CACHE names a file, is
// read from and appended to that file (one line per entry:
// "kernel Lx Ly Lz Lt nrhs prec gpu block ms").
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "internal.h"

namespace mg {

namespace {
std::mutex g_tune_mutex;
std::map<std::string, int> g_table;
bool g_loaded = false;

std::string gpu_name() {
  int dev = 0;
  MG_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp p;
  MG_CUDA(cudaGetDeviceProperties(&p, dev));
  std::string n = p.name;
  for (char& ch : n)
    if (ch == ' ') ch = '_';
  return n;
}

std::string key_of(const TuneKey& k) {
  std::ostringstream o;
  o << k.kernel << ' ' << k.dims[0] << ' ' << k.dims[1] << ' ' << k.dims[2] << ' ' << k.dims[3] << ' ' << k.nrhs << ' '
    << k.prec << ' ' << gpu_name();
  return o.str();
}

void load_file() {
  g_loaded = true;
  const char* path = std::getenv("MGCLOVER_TUNE_CACHE");
  if (!path) return;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream in(line);
    std::string kernel, gpu;
    int d[4], nrhs, prec, block;
    double ms;
    if (in >> kernel >> d[0] >> d[1] >> d[2] >> d[3] >> nrhs >> prec >> gpu >> block >> ms) {
      std::ostringstream o;
      o << kernel << ' ' << d[0] << ' ' << d[1] << ' ' << d[2] << ' ' << d[3] << ' ' << nrhs << ' ' << prec << ' ' << gpu;
      g_table[o.str()] = block;
    }
  }
}

void save_line(const std::string& key, int block, double ms) {
  const char* path = std::getenv("MGCLOVER_TUNE_CACHE");
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << ' ' << block << ' ' << ms << '\n';
}
}  // namespace

int tuned_block(const TuneKey& k, const std::vector<int>& candidates, const std::function<void(int)>& launch,
                cudaStream_t s) {
  if (candidates.empty()) raise(MG_ERR_ARG, "no tuning candidates");
  const std::string key = key_of(k);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    if (!g_loaded) load_file();
    auto it = g_table.find(key);
    if (it != g_table.end()) return it->second;
  }
  cudaEvent_t e0, e1;
  MG_CUDA(cudaEventCreate(&e0));
  MG_CUDA(cudaEventCreate(&e1));
  int best = candidates[0];
  float best_ms = 1e30f;
  for (int b : candidates) {
    launch(b);  // warm-up
    MG_CUDA(cudaEventRecord(e0, s));
    constexpr int reps = 3;
    for (int r = 0; r < reps; r++) launch(b);
    MG_CUDA(cudaEventRecord(e1, s));
    MG_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    MG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    ms /= reps;
    if (ms < best_ms) {
      best_ms = ms;
      best = b;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_table[key] = best;
  save_line(key, best, best_ms);
  return best;
}

int tune_entries() {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  return (int)g_table.size();
}

}  // namespace mg
