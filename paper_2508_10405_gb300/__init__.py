"""GB300 (sm_103a) multiparameter LSRTM operators: Born modelling L, its exact
adjoint L^T (migration), PSF probes and a CGNR driver for the first-order
velocity-pressure acoustic system parametrised by (dln Vp, dln Ip).

The compute path is the CUDA library built from csrc/ (liblsrtm.so, C ABI in
include/lsrtm.h); this package only marshals arguments to it."""
from .binding import (BAND_BF16, BAND_FP16, BAND_FP32, EXPORTS, PLAN_BATCHED, PLAN_PLAIN, RECON_AUTO,
                      RECON_BOUNDARY, RECON_CHECKPOINT, Lsrtm, LsrtmError, born_op, load_library)

__all__ = ["Lsrtm", "LsrtmError", "born_op", "load_library", "EXPORTS", "BAND_FP32",
           "BAND_BF16", "BAND_FP16", "PLAN_BATCHED", "PLAN_PLAIN", "RECON_BOUNDARY", "RECON_CHECKPOINT",
           "RECON_AUTO"]
