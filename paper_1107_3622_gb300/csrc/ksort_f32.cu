// Kernels and launchers of libksort for float keys.
#include "ksort_launch.cuh"

template struct ksort::Launcher<float>;
