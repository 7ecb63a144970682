// prof.cu -- optional per-kernel CUDA-event timing of a grid's launches.
#include <stdlib.h>

#include "phl_internal.cuh"

namespace phl {

const char *kclass_name(int c) {
  static const char *names[KC_COUNT] = {"prim",         "flag_raw",     "flag_dilate", "flux_x",
                                        "flux_y",       "flux_z",       "emf",         "update_cells",
                                        "update_faces", "dt",           "set_scalar",  "stage_mixed",
                                        "flux_update",  "sph_prim",     "sph_flux",    "sph_emf",
                                        "sph_update_faces", "sph_update_cells", "sph_dt"};
  return (c >= 0 && c < KC_COUNT) ? names[c] : "?";
}

cudaError_t Prof::begin(int c, cudaStream_t s) {
  if (!on) return cudaSuccess;
  if (cap == 0) {
    cap = 4096;
    ev = (cudaEvent_t *)calloc(2 * (size_t)cap, sizeof(cudaEvent_t));
    cls = (int *)calloc((size_t)cap, sizeof(int));
    for (int i = 0; i < 2 * cap; ++i) {
      cudaError_t e = cudaEventCreate(&ev[i]);
      if (e != cudaSuccess) return e;
    }
  }
  if (used == cap) {
    cudaError_t e = fold();
    if (e != cudaSuccess) return e;
  }
  cls[used] = c;
  cur = used;
  return cudaEventRecord(ev[2 * used], s);
}

cudaError_t Prof::end(cudaStream_t s) {
  if (!on || cur < 0) return cudaSuccess;
  cudaError_t e = cudaEventRecord(ev[2 * cur + 1], s);
  cur = -1;
  ++used;
  return e;
}

cudaError_t Prof::fold() {
  for (int i = 0; i < used; ++i) {
    cudaError_t e = cudaEventSynchronize(ev[2 * i + 1]);
    if (e != cudaSuccess) return e;
    float t = 0.f;
    e = cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
    if (e != cudaSuccess) return e;
    ms[cls[i]] += t;
    cnt[cls[i]] += 1;
  }
  used = 0;
  return cudaSuccess;
}

void Prof::release() {
  if (ev) {
    for (int i = 0; i < 2 * cap; ++i) cudaEventDestroy(ev[i]);
    free(ev);
    free(cls);
  }
  ev = nullptr;
  cls = nullptr;
  cap = used = 0;
}

}  // namespace phl
