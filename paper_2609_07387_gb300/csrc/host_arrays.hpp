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
  std::vector<double> Pd;                                // [nd][Kd][Md][N]
  std::vector<double> Msi;                               // P3/P4: [K(K+1)/2][N]
  std::vector<double> psib;                              // P3/P4: [K-3][N]
  std::vector<double> fq;                                // [nq][10][F] x-x_L, x-x_R', n, |dS|
  std::vector<double> fpen;                              // [F] (0 on boundary faces)
  std::vector<int8_t> fkind;                             // [F] -1 interior, else the boundary kind
  std::vector<uint8_t> dvalid;                           // [N] bit s: directional candidate s exists
};

}  // namespace ucns
