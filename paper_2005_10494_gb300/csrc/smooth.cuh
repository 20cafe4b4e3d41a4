// Host-side shape check of the smoothing launch (smooth.cu).
#pragma once

namespace mcd {

// nullptr when smooth_argmax can launch n_scen grids of g1 x g2, else the
// reason it cannot.
const char* smooth_shape_error(int n_scen, int g1, int g2);

}  // namespace mcd
