"""GB300-native differentiable tile-based 3D Gaussian splatting for
LiDAR-camera spatiotemporal calibration (3DGS-Calib, arXiv 2403.11577).

Submodules:
  scenes  - seeded synthetic inputs (no method arithmetic)
  capi    - ctypes binding of the C-ABI library libgs3dcalib.so
  render  - batch planning, workspace, torch.autograd.Function wrapper,
            CUDA-graph calibration step
  autotune - tile / shared-memory batch autotuner
The CUDA library is loaded lazily on first use of `capi`; importing the
package never touches the GPU.
"""
__version__ = "0.1.0"
