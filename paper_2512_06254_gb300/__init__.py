"""GB300 (sm_103a) implementation of the FIP-TOI hot path.

Per snapshot: TOI 2-D imaging (plane fit, convolutional gridding, inverse
FFT, grid correction, reduced SIN re-projection) and FITrig's tLISI tile
statistic; over the stream: candidate search on the tLISI cube.  The
computation lives in the CUDA library libtoi (C ABI, include/toi.h); this
package holds its ctypes binding, the build script and the seeded input
generator.
"""
from .binding import (Plan, Stream, ToiError, tlisi_candidates, lib, config_default,  # noqa: F401
                      TOI_OK, TOI_ERR_ARG, TOI_ERR_CUDA, TOI_ERR_OOM, TOI_ERR_EMPTY,
                      TOI_ERR_TIMEOUT, TOI_ERR_UNSUPPORTED, TOI_ERR_RANGE, TOI_VIS_C64,
                      TOI_VIS_C16_CHANSCALE, TOI_CAND_PERIODIC, TOI_CAND_NONPERIODIC,
                      BUF_GRID, BUF_TILTED, BUF_SNAP, BUF_RING)
