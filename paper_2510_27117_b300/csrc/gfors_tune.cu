// gfors_tune.cu -- autotuner entry points and its JSON cache (host code).
//
// The batched PDHG path processes rows (dual step) and columns (primal step)
// in five length buckets; the number of threads per row / column of each
// bucket is the tunable.  gfors_autotune times the choices on the device and
// keeps the fastest, or takes them from a cache file keyed by the device name
// and the batch's shape class.  Cache format: one JSON object, one entry per
// line:  "<key>": {"rows": [l0, l1, l2, l3, l4], "cols": [l0, l1, l2, l3, l4]}
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <fstream>
#include <sstream>
#include <string>
#include <utility>
#include <vector>

#include "internal.cuh"

cudaError_t gf_tune_lanes(GfCtx* h, int32_t lanes_out[10]);

namespace {

bool valid_lanes(const int32_t* l) {
  for (int k = 0; k < 10; ++k)
    if (l[k] != 1 && l[k] != 2 && l[k] != 4 && l[k] != 8 && l[k] != 16 && l[k] != 32)
      return false;
  return true;
}

using Entry = std::pair<std::string, std::vector<int32_t>>;

// Entries of a cache file written by write_cache (missing file: none).
std::vector<Entry> read_cache(const char* path) {
  std::vector<Entry> out;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t q0 = line.find('"');
    if (q0 == std::string::npos) continue;
    const size_t q1 = line.find('"', q0 + 1);
    const size_t r = line.find("\"rows\": [");
    const size_t c = line.find("\"cols\": [");
    if (q1 == std::string::npos || r == std::string::npos || c == std::string::npos) continue;
    std::vector<int32_t> l(10, 0);
    if (sscanf(line.c_str() + r + 9, "%d, %d, %d, %d, %d", &l[0], &l[1], &l[2], &l[3],
               &l[4]) != 5)
      continue;
    if (sscanf(line.c_str() + c + 9, "%d, %d, %d, %d, %d", &l[5], &l[6], &l[7], &l[8],
               &l[9]) != 5)
      continue;
    if (!valid_lanes(l.data())) continue;
    out.emplace_back(line.substr(q0 + 1, q1 - q0 - 1), l);
  }
  return out;
}

bool write_cache(const char* path, const std::vector<Entry>& es) {
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream f(tmp, std::ios::trunc);
    if (!f) return false;
    f << "{\n";
    for (size_t u = 0; u < es.size(); ++u) {
      const std::vector<int32_t>& l = es[u].second;
      f << "  \"" << es[u].first << "\": {\"rows\": [" << l[0] << ", " << l[1] << ", " << l[2]
        << ", " << l[3] << ", " << l[4] << "], \"cols\": [" << l[5] << ", " << l[6] << ", "
        << l[7] << ", " << l[8] << ", " << l[9] << "]}" << (u + 1 < es.size() ? "," : "")
        << "\n";
    }
    f << "}\n";
    if (!f) return false;
  }
  return rename(tmp.c_str(), path) == 0;
}

int log2_class(int64_t v) { return v <= 0 ? -1 : (int)std::floor(std::log2((double)v)); }

std::string shape_key(GfCtx* h) {
  cudaDeviceProp pr;
  std::string dev = "unknown";
  if (cudaGetDeviceProperties(&pr, h->dev) == cudaSuccess) dev = pr.name;
  else cudaGetLastError();
  for (char& ch : dev)
    if (ch == '"' || ch == '\\' || (unsigned char)ch < 32) ch = '_';
  std::ostringstream k;
  k << dev << "|N" << log2_class(h->N) << "|M" << log2_class(h->M) << "|K"
    << log2_class(h->nnzK) << "|r";
  for (size_t b = 0; b < h->rb.size(); ++b) k << (b ? "." : "") << log2_class(h->rb[b].count);
  k << "|c";
  for (size_t b = 0; b < h->cb.size(); ++b) k << (b ? "." : "") << log2_class(h->cb[b].count);
  return k.str();
}

void drop_graphs(GfCtx* h) {
  for (int q = 0; q < 2; ++q) {
    if (h->g_iter2[q]) {
      cudaGraphExecDestroy(h->g_iter2[q]);
      h->g_iter2[q] = nullptr;
    }
    if (h->g_light2[q]) {
      cudaGraphExecDestroy(h->g_light2[q]);
      h->g_light2[q] = nullptr;
    }
  }
}

void apply_lanes(GfCtx* h, const int32_t* l) {
  for (size_t k = 0; k < h->rb.size() && k < 5; ++k) h->rb[k].lanes = l[k];
  for (size_t k = 0; k < h->cb.size() && k < 5; ++k) h->cb[k].lanes = l[5 + k];
  drop_graphs(h);
  h->struct_version++;                  // a cached whole-run graph is rebuilt
}

}  // namespace

extern "C" gfors_status gfors_tune_cache_lookup(const char* path, const char* key,
                                                int32_t lanes[10], int32_t* found) {
  if (!path || !key || !lanes || !found) return GFORS_E_ARG;
  *found = 0;
  for (const Entry& e : read_cache(path))
    if (e.first == key) {
      for (int k = 0; k < 10; ++k) lanes[k] = e.second[k];
      *found = 1;
    }
  return GFORS_OK;
}

extern "C" gfors_status gfors_tune_cache_store(const char* path, const char* key,
                                               const int32_t lanes[10]) {
  if (!path || !key || !lanes || !valid_lanes(lanes)) return GFORS_E_ARG;
  for (const char* p = key; *p; ++p)
    if (*p == '"' || *p == '\\' || (unsigned char)*p < 32) return GFORS_E_ARG;
  std::vector<Entry> es = read_cache(path);
  std::vector<int32_t> l(lanes, lanes + 10);
  bool put = false;
  for (Entry& e : es)
    if (e.first == key) { e.second = l; put = true; }
  if (!put) es.emplace_back(key, l);
  return write_cache(path, es) ? GFORS_OK : GFORS_E_ARG;
}

extern "C" gfors_status gfors_tune_key(gfors_handle h, char* buf, size_t len) {
  if (!h || !buf || len == 0) return GFORS_E_ARG;
  const std::string k = shape_key(h);
  if (k.size() + 1 > len) return gf_fail(h, GFORS_E_ARG, "gfors_tune_key: buffer too small");
  memcpy(buf, k.c_str(), k.size() + 1);
  return GFORS_OK;
}

extern "C" gfors_status gfors_set_lanes(gfors_handle h, const int32_t lanes[10]) {
  if (!h) return GFORS_E_ARG;
  if (h->failed) return GFORS_E_STATE;
  if (!lanes || !valid_lanes(lanes))
    return gf_fail(h, GFORS_E_ARG, "lanes must be 1, 2, 4, 8, 16 or 32");
  apply_lanes(h, lanes);
  return GFORS_OK;
}

extern "C" gfors_status gfors_get_lanes(gfors_handle h, int32_t lanes[10]) {
  if (!h || !lanes) return GFORS_E_ARG;
  for (int k = 0; k < 5; ++k) {
    lanes[k] = k < (int)h->rb.size() ? h->rb[k].lanes : 0;
    lanes[5 + k] = k < (int)h->cb.size() ? h->cb[k].lanes : 0;
  }
  return GFORS_OK;
}

extern "C" gfors_status gfors_autotune(gfors_handle h, const char* cache_path,
                                       int32_t out_lanes[10], int32_t* hit) {
  if (!h) return GFORS_E_ARG;
  if (h->failed) return GFORS_E_STATE;
  int32_t l[10];
  int32_t found = 0;
  const std::string key = shape_key(h);
  if (cache_path) gfors_tune_cache_lookup(cache_path, key.c_str(), l, &found);
  if (found) {
    apply_lanes(h, l);
  } else {
    cudaError_t e = gf_tune_lanes(h, l);
    if (e != cudaSuccess) return gf_cuda(h, e, "gfors_autotune");
    drop_graphs(h);
    if (cache_path && gfors_tune_cache_store(cache_path, key.c_str(), l) != GFORS_OK)
      return gf_fail(h, GFORS_E_ARG, std::string("cannot write tuning cache ") + cache_path);
  }
  if (out_lanes)
    for (int k = 0; k < 10; ++k) out_lanes[k] = l[k];
  if (hit) *hit = found;
  return GFORS_OK;
}
