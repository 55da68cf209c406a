"""GB300-native (sm_103a CUDA) DiffCloud mesh-to-point-cloud loss.

The loss of DiffCloud (Sundaresan et al. 2022, Sec. III): area-weighted sampling of each
simulated mesh frame (Sec. III-B, Eq. 3), brute-force Chamfer distance to the observed cloud
(Eq. 1 / Eq. 2), and its gradient with respect to every mesh vertex (Eq. 4). The compute
runs in libdiffcloud.so (include/diffcloud.h); this package is its Python binding.
"""
from ._lib import (BIDIR_MEAN, UNIDIR_SUM, DCError, dc_chamfer_bwd, dc_chamfer_fwd,
                   dc_loss_traj, dc_loss_traj_bwd, dc_sample, dc_workspace_size, lib,
                   lib_path, launch_count, last_error)

__all__ = ["BIDIR_MEAN", "UNIDIR_SUM", "DCError", "dc_chamfer_bwd", "dc_chamfer_fwd",
           "dc_loss_traj", "dc_loss_traj_bwd", "dc_sample", "dc_workspace_size", "lib",
           "lib_path", "launch_count", "last_error"]
