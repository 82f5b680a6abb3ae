// Host staging buffers of ucns_precompute, structure-of-arrays in the
// internal cell order, uploaded once to the device.
#pragma once

#include <cstdint>
#include <vector>

namespace ucns {

struct HostArrays {
  std::vector<double> vol, inv_vol, inv_h, dtlen, mom;  // mom [6][N]
  std::vector<int32_t> sc;                               // [Mc][N]
  std::vector<double> Pc;                                // [K][Mc][N]
  std::vector<int32_t> sd;                               // [nd][Md][N]
  std::vector<double> Pd;                                // [nd][3][Md][N]
  std::vector<double> fq;                                // [nq][10][F] x-x_L, x-x_R', n, |dS|
  std::vector<double> fpen;                              // [F]
};

}  // namespace ucns
