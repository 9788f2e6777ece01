// Autotuner: measures, on the current GPU, the window size up to which the
// direct method beats the blocked van Herk/Gil-Werman method, per pixel type
// and per pass -- the crossovers w_x^0 / w_y^0 of the paper's section 5.3,
// which the paper measured on an ARM CPU (59 and 69) and which differ on a
// GPU -- and, per pixel type, whether the pass along x runs faster inside the
// fused kernel or through the standalone transpose kernels (section 5.2.1's
// form), the rows per warp of the pass along x (2 or 4, on a 4096 x 2048
// image), the fused kernel's tile shape per pixel type and direct-method
// window class (2048 x 2048 images), and the tile height of the pass along
// y per pixel type and window class (4096 x 4096 images; the paper's
// section 5.3 likewise sets its parameters by measuring on the target).
// Results persist as a small JSON file keyed by the device.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/morph.h"
#include "morph_internal.h"
#include "plan.h"

namespace morph {
namespace {

constexpr int kTuneW = 2048, kTuneH = 2048;  // synthetic image for the timings
constexpr int kReps = 5;

std::string device_key() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p;
  memset(&p, 0, sizeof(p));
  cudaGetDeviceProperties(&p, dev);
  int drv = 0;
  cudaDriverGetVersion(&drv);
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|sm%d%d|%dSM|drv%d|v6", p.name, p.major, p.minor, p.multiProcessorCount, drv);
  return buf;
}

// Mean GPU time (ms) of one call in the planned form under the current
// tuning.  The calls are captured into a CUDA graph and the graph is timed,
// so that host-side launch cost (which can exceed the kernel's own time on a
// small image) does not enter the comparison.
float time_planned(const FusedLaunch& L, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  constexpr int kCalls = 8;
  if (launch_planned(L, st) != MORPH_OK) return 1e30f;  // set-up outside the capture
  if (cudaStreamSynchronize(st) != cudaSuccess) return 1e30f;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return 1e30f;
  bool ok = true;
  for (int i = 0; i < kCalls; ++i) ok = ok && launch_planned(L, st) == MORPH_OK;
  if (cudaStreamEndCapture(st, &graph) != cudaSuccess || !ok) {
    if (graph) cudaGraphDestroy(graph);
    return 1e30f;
  }
  float best = 1e30f;
  if (cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
    std::vector<float> t;
    for (int r = 0; r < kReps + 1; ++r) {
      cudaEventRecord(e0, st);
      cudaGraphLaunch(exec, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r) t.push_back(ms / kCalls);  // the first replay warms up
    }
    if (!t.empty()) {
      std::sort(t.begin(), t.end());
      best = t[t.size() / 2];
    }
    cudaGraphExecDestroy(exec);
  }
  cudaGraphDestroy(graph);
  return best;
}
float time_launch(const FusedLaunch& L, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  return time_planned(L, st, e0, e1);
}

bool load_cache(const char* path, const std::string& key, Tuning* t) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char buf[4096];
  const size_t n = fread(buf, 1, sizeof(buf) - 1, f);
  fclose(f);
  buf[n] = 0;
  const std::string s(buf);
  const std::string kq = "\"device\": \"" + key + "\"";
  if (s.find(kq) == std::string::npos) return false;
  int v[4];
  const char* p = strstr(buf, "\"cross\": [");
  if (!p || sscanf(p, "\"cross\": [%d, %d, %d, %d]", &v[0], &v[1], &v[2], &v[3]) != 4) return false;
  for (int x : v)
    if (x < 0 || x > 100000) return false;
  t->cross_row[0] = v[0];
  t->cross_col[0] = v[1];
  t->cross_row[1] = v[2];
  t->cross_col[1] = v[3];
  int xp[2] = {0, 0};
  const char* q = strstr(buf, "\"xpass\": [");
  if (q && sscanf(q, "\"xpass\": [%d, %d]", &xp[0], &xp[1]) == 2) {
    t->xpass_transpose[0] = xp[0] == 1;
    t->xpass_transpose[1] = xp[1] == 1;
  }
  int rr[2];
  const char* r = strstr(buf, "\"rowv_rows\": [");
  if (r && sscanf(r, "\"rowv_rows\": [%d, %d]", &rr[0], &rr[1]) == 2)
    for (int i = 0; i < 2; ++i)
      if (rr[i] == 2 || rr[i] == 4 || rr[i] == 8) t->rowv_rr[i] = rr[i];
  int fc[16];
  const char* f1 = strstr(buf, "\"fused_cfg\": [");
  if (f1 && sscanf(f1, "\"fused_cfg\": [%d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d]", &fc[0],
                   &fc[1], &fc[2], &fc[3], &fc[4], &fc[5], &fc[6], &fc[7], &fc[8], &fc[9], &fc[10], &fc[11], &fc[12],
                   &fc[13], &fc[14], &fc[15]) == 16)
    for (int i = 0; i < 16; ++i)
      t->fused_cfg_tuned[i / 8][(i / 2) % 4][i % 2] = fc[i] >= 0 && fc[i] < kNumTileCfg ? fc[i] : -1;
  int cf[10];
  const char* f2 = strstr(buf, "\"colv_family\": [");
  if (f2 && sscanf(f2, "\"colv_family\": [%d, %d, %d, %d, %d, %d, %d, %d, %d, %d]", &cf[0], &cf[1], &cf[2], &cf[3],
                   &cf[4], &cf[5], &cf[6], &cf[7], &cf[8], &cf[9]) == 10)
    for (int i = 0; i < 10; ++i) t->colv_fam_tuned[i / 5][i % 5] = cf[i] >= 0 && cf[i] < kColvFamilies ? cf[i] : -1;
  return true;
}

bool save_cache(const char* path, const std::string& key, const Tuning& t) {
  FILE* f = fopen(path, "w");
  if (!f) return false;
  fprintf(f,
          "{\"device\": \"%s\", \"cross\": [%d, %d, %d, %d], \"order\": \"u8 x, u8 y, u16 x, u16 y\", "
          "\"xpass\": [%d, %d], \"rowv_rows\": [%d, %d], "
          "\"fused_cfg\": [%d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d], "
          "\"fused_cfg_order\": \"u8 windows <=3 <=5 <=7 <=9, each for images below 8 Mpixels and larger; "
          "u16 the same; tile configuration or -1\", "
          "\"colv_family\": [%d, %d, %d, %d, %d, %d, %d, %d, %d, %d], "
          "\"colv_family_order\": \"u8 windows <=24 <=40 <=76 <=114 above, u16 the same; 0 rule, 1-3 multiples of "
          "the window, 4-6 64/128/256 rows\"}\n",
          key.c_str(), t.cross_row[0], t.cross_col[0], t.cross_row[1], t.cross_col[1], t.xpass_transpose[0],
          t.xpass_transpose[1], t.rowv_rr[0], t.rowv_rr[1], t.fused_cfg_tuned[0][0][0], t.fused_cfg_tuned[0][0][1],
          t.fused_cfg_tuned[0][1][0], t.fused_cfg_tuned[0][1][1], t.fused_cfg_tuned[0][2][0],
          t.fused_cfg_tuned[0][2][1], t.fused_cfg_tuned[0][3][0], t.fused_cfg_tuned[0][3][1],
          t.fused_cfg_tuned[1][0][0], t.fused_cfg_tuned[1][0][1], t.fused_cfg_tuned[1][1][0],
          t.fused_cfg_tuned[1][1][1], t.fused_cfg_tuned[1][2][0], t.fused_cfg_tuned[1][2][1],
          t.fused_cfg_tuned[1][3][0], t.fused_cfg_tuned[1][3][1], t.colv_fam_tuned[0][0], t.colv_fam_tuned[0][1],
          t.colv_fam_tuned[0][2], t.colv_fam_tuned[0][3], t.colv_fam_tuned[0][4], t.colv_fam_tuned[1][0],
          t.colv_fam_tuned[1][1], t.colv_fam_tuned[1][2], t.colv_fam_tuned[1][3], t.colv_fam_tuned[1][4]);
  return fclose(f) == 0;
}

}  // namespace
}  // namespace morph

using namespace morph;

extern "C" int morph_autotune(const char* cache_path) {
  const std::string key = device_key();
  Tuning& t = tuning();
  if (cache_path && load_cache(cache_path, key, &t)) {
    t.from_autotune = 1;
    return MORPH_OK;
  }
  void *src = nullptr, *dst = nullptr;
  const size_t pitch = kTuneW * 2;
  if (cudaMalloc(&src, pitch * kTuneH) != cudaSuccess) return MORPH_ERR_NOMEM;
  if (cudaMalloc(&dst, pitch * kTuneH) != cudaSuccess) {
    cudaFree(src);
    return MORPH_ERR_NOMEM;
  }
  cudaMemset(src, 0x5A, pitch * kTuneH);
  cudaStream_t st;
  cudaEvent_t e0, e1;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int forced0 = t.forced_cfg[0], forced1 = t.forced_cfg[1];
  int rc = MORPH_OK;
  // Candidate windows; the direct method needs no minimum, the blocked one w >= 8.
  const int cands[] = {8, 9, 11, 13, 15, 17, 21, 25, 31, 41, 51, 63};
  int found[2][2] = {{7, 7}, {7, 7}};  // [type][axis 0: pass along x, 1: along y]
  for (int e = 0; e < 2 && rc == MORPH_OK; ++e) {
    for (int axis = 0; axis < 2 && rc == MORPH_OK; ++axis) {
      for (int w : cands) {  // direct for w <= 7 always (the blocked method needs w >= 8)
        FusedLaunch L;
        memset(&L, 0, sizeof(L));
        L.esz = e + 1;
        L.op = 0;
        L.src = src;
        L.dst = dst;
        L.sp = L.dp = static_cast<long long>(pitch);
        L.W = kTuneW;
        L.H = kTuneH;
        L.wx = axis == 0 ? w : 1;  // a 1-D window: only the measured pass runs
        L.wy = axis == 0 ? 1 : w;
        L.ax = L.wx / 2;
        L.ay = L.wy / 2;
        t.cross_row[e] = t.cross_col[e] = 1 << 30;  // direct
        const float td = time_launch(L, st, e0, e1);
        t.cross_row[e] = t.cross_col[e] = 0;  // blocked
        const float tb = time_launch(L, st, e0, e1);
        if (td >= 1e29f || tb >= 1e29f) {
          rc = MORPH_ERR_CUDA;
          break;
        }
        if (td <= tb)
          found[e][axis] = w;
        else
          break;
      }
    }
  }
  for (int e = 0; e < 2; ++e) {
    t.cross_row[e] = found[e][0];
    t.cross_col[e] = found[e][1];
  }
  t.forced_cfg[0] = forced0;
  t.forced_cfg[1] = forced1;
  // The pass along x: fused (register transposes) or through the transpose
  // kernels, timed on a small and a large 1-D window along x.
  for (int e = 0; e < 2 && rc == MORPH_OK; ++e) {
    float tf = 0, tt = 0;
    for (int w : {15, 101}) {
      FusedLaunch L;
      memset(&L, 0, sizeof(L));
      L.esz = e + 1;
      L.src = src;
      L.dst = dst;
      L.sp = L.dp = static_cast<long long>(pitch);
      L.W = kTuneW;
      L.H = kTuneH;
      L.wx = w;
      L.ax = w / 2;
      L.wy = 1;
      t.xpass_transpose[e] = 0;
      tf += time_planned(L, st, e0, e1);
      t.xpass_transpose[e] = 1;
      tt += time_planned(L, st, e0, e1);
    }
    if (tf >= 1e29f || tt >= 1e29f) rc = MORPH_ERR_CUDA;
    t.xpass_transpose[e] = tt < tf ? 1 : 0;
  }
  cudaFree(src);
  cudaFree(dst);
  src = dst = nullptr;
  // Rows per warp of the pass along x, on a 4096 x 2048 image (as many row
  // bands as the large images it serves).
  constexpr int kShapeW = 4096, kShapeH = 2048;
  const size_t spitch = kShapeW * 2;
  if (rc == MORPH_OK && (cudaMalloc(&src, spitch * kShapeH) != cudaSuccess ||
                         cudaMalloc(&dst, spitch * kShapeH) != cudaSuccess))
    rc = MORPH_ERR_NOMEM;
  if (rc == MORPH_OK) cudaMemset(src, 0x3C, spitch * kShapeH);
  for (int e = 0; e < 2 && rc == MORPH_OK; ++e) {
    FusedLaunch L;
    memset(&L, 0, sizeof(L));
    L.esz = e + 1;
    L.src = src;
    L.dst = dst;
    L.sp = L.dp = static_cast<long long>(spitch);
    L.W = kShapeW;
    L.H = kShapeH;
    // pass along x: 2 or 4 rows per warp
    L.wy = 1;
    L.ay = 0;
    L.wx = 101;
    L.ax = 50;
    float best = 1e30f;
    int best_r = 2;
    for (int rr : {2, 4}) {
      if (rc != MORPH_OK) break;
      t.rowv_rr[e] = rr;
      const float ms = time_planned(L, st, e0, e1);
      if (ms >= 1e29f) rc = MORPH_ERR_CUDA;
      if (ms < best) {
        best = ms;
        best_r = rr;
      }
    }
    t.rowv_rr[e] = best_r;
  }
  // Tile height of the pass along y per window class, on a 4096 x 4096
  // image (the size class the measured heights serve): each of the heights
  // the planner can be given, the built-in rule among them; the fastest is
  // kept (ties to the rule).
  cudaFree(src);
  cudaFree(dst);
  src = dst = nullptr;
  constexpr int kBigH = 4096;
  if (rc == MORPH_OK && (cudaMalloc(&src, spitch * kBigH) != cudaSuccess ||
                         cudaMalloc(&dst, spitch * kBigH) != cudaSuccess))
    rc = MORPH_ERR_NOMEM;
  if (rc == MORPH_OK) cudaMemset(src, 0x3C, spitch * kBigH);
  const int colv_windows[5] = {15, 31, 51, 101, 127};
  for (int e = 0; e < 2 && rc == MORPH_OK; ++e) {
    for (int c = 0; c < 5 && rc == MORPH_OK; ++c) {
      FusedLaunch L;
      memset(&L, 0, sizeof(L));
      L.esz = e + 1;
      L.src = src;
      L.dst = dst;
      L.sp = L.dp = static_cast<long long>(spitch);
      L.W = kShapeW;
      L.H = kBigH;
      L.wx = 1;
      L.ax = 0;
      L.wy = colv_windows[c];
      L.ay = L.wy / 2;
      float best = 1e30f;
      int best_f = 0;
      for (int fam = 0; fam < kColvFamilies && rc == MORPH_OK; ++fam) {
        t.colv_fam_tuned[e][c] = fam;
        const float ms = time_planned(L, st, e0, e1);
        if (ms >= 1e29f) rc = MORPH_ERR_CUDA;
        if (ms < best * 0.98f) {  // another height must beat the rule clearly
          best = ms;
          best_f = fam;
        }
      }
      t.colv_fam_tuned[e][c] = best_f;
    }
  }
  // Tile shape of the fused kernel per direct-method window class (square
  // windows 3, 5, 7, 9) and size class: every shape that fits, the fastest
  // kept; first on this 4096 x 4096 image, then on a 2048 x 2048 one.
  const int fused_windows[4] = {3, 5, 7, 9};
  auto tune_shapes = [&](int sc, int W, int H, long long sp) {
    for (int e = 0; e < 2 && rc == MORPH_OK; ++e) {
      for (int c = 0; c < 4 && rc == MORPH_OK; ++c) {
        FusedLaunch L;
        memset(&L, 0, sizeof(L));
        L.esz = e + 1;
        L.src = src;
        L.dst = dst;
        L.sp = L.dp = sp;
        L.W = W;
        L.H = H;
        L.wx = L.wy = fused_windows[c];
        L.ax = L.ay = L.wx / 2;
        FusedLaunch P = L;
        if (!plan_single(&P) || P.vhgw_col || P.vhgw_row) {
          t.fused_cfg_tuned[e][c][sc] = -1;  // not a direct-method window at the crossovers found
          continue;
        }
        float best = 1e30f;
        int best_c = -1;
        for (int cfg = 0; cfg < kNumTileCfg && rc == MORPH_OK; ++cfg) {
          FusedLaunch Q = P;
          Q.cfg = cfg;
          const int b = fused_smem_bytes(Q);
          if (b <= 0 || b > kMaxSmemBytes) continue;
          t.fused_cfg_tuned[e][c][sc] = cfg;
          const float ms = time_planned(L, st, e0, e1);
          if (ms >= 1e29f) rc = MORPH_ERR_CUDA;
          if (ms < best) {
            best = ms;
            best_c = cfg;
          }
        }
        t.fused_cfg_tuned[e][c][sc] = best_c;
      }
    }
  };
  if (rc == MORPH_OK) tune_shapes(1, kShapeW, kBigH, static_cast<long long>(spitch));
  cudaFree(src);
  cudaFree(dst);
  src = dst = nullptr;
  if (rc == MORPH_OK && (cudaMalloc(&src, pitch * kTuneH) != cudaSuccess ||
                         cudaMalloc(&dst, pitch * kTuneH) != cudaSuccess))
    rc = MORPH_ERR_NOMEM;
  if (rc == MORPH_OK) cudaMemset(src, 0x66, pitch * kTuneH);
  if (rc == MORPH_OK) tune_shapes(0, kTuneW, kTuneH, static_cast<long long>(pitch));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (src) cudaFree(src);
  if (dst) cudaFree(dst);
  if (rc != MORPH_OK) {
    reset_tuning_defaults();
    return rc;
  }
  t.from_autotune = 1;
  if (cache_path && !save_cache(cache_path, key, t)) return MORPH_ERR_ARG;
  return MORPH_OK;
}
