// Kernel instances for f64 values (double vectors and accumulation).
#include "spmv_launch.cuh"

namespace pjds {

int pjds_launch_f64(const pjds_dev *A, const void *x, void *y, const LaunchCfg &c, cudaStream_t s) {
  return launch_pjds<double, double>(A, x, y, c, s);
}

int ellr_launch_f64(const ellr_dev *A, const void *x, void *y, int nt, cudaStream_t s) {
  return launch_ellr<double, double>(A, x, y, nt, s);
}

int staged_wait_selftest(int which, cudaStream_t s) {
  dev::staged_wait_selftest_kernel<<<1, 32, 0, s>>>(which);
  return check_launch("wait self-test launch");
}

int staged_status_f64(int *out, bool clear, cudaStream_t s) {
  return (int)dev::staged_status(out, clear, s);
}

int check_word_f64(unsigned long long *w, bool clear, cudaStream_t s) { return check_word_here<>(w, clear, s); }

}  // namespace pjds
