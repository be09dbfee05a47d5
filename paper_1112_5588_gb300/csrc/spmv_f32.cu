// Kernel instances for f32 values (float vectors and accumulation).
#include "spmv_launch.cuh"

namespace pjds {

int pjds_launch_f32(const pjds_dev *A, const void *x, void *y, const LaunchCfg &c, cudaStream_t s) {
  return launch_pjds<float, float>(A, x, y, c, s);
}

int ellr_launch_f32(const ellr_dev *A, const void *x, void *y, int nt, cudaStream_t s) {
  return launch_ellr<float, float>(A, x, y, nt, s);
}

int staged_status_f32(int *out, bool clear, cudaStream_t s) {
  return (int)dev::staged_status(out, clear, s);
}

int check_word_f32(unsigned long long *w, bool clear, cudaStream_t s) { return check_word_here<>(w, clear, s); }

}  // namespace pjds
