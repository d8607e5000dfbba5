// The library-owned NSSG index (the opaque ssg_graph of include/ssg.h).
#pragma once

#include <vector>

#include "common.cuh"

struct ssg_graph {
  int64_t n = 0;
  int32_t d = 0, R = 0, n_nav = 0;
  double alpha = 0;
  int32_t* adj = nullptr;      // device [n][R], -1 padded (the paper's n x m matrix, Sec. 5.4)
  int32_t* deg = nullptr;      // device [n]
  int32_t* nav_dev = nullptr;  // device [n_nav]
  std::vector<int32_t> nav_host;
  float* base_owned = nullptr;  // device copy of the base when built from host vectors
  // Byte copy of the base rows [n][rows_ld] when the data are integers 0..255, read by
  // searches given the base it was made from (rows_src) instead of the float rows.
  uint8_t* rows_u8 = nullptr;
  int32_t rows_ld = 0;
  const float* rows_src = nullptr;
  ~ssg_graph() {
    if (rows_u8) cudaFree(rows_u8);
    if (adj) cudaFree(adj);
    if (deg) cudaFree(deg);
    if (nav_dev) cudaFree(nav_dev);
    if (base_owned) cudaFree(base_owned);
  }
};
