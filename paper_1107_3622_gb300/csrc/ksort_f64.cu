// Kernels and launchers of libksort for double keys.
#include "ksort_launch.cuh"

template struct ksort::Launcher<double>;
