"""GB300 (sm_103a) implementation of the Shan-Chen bubble-merging lattice
Boltzmann hot path of arXiv 1708.01608: fused collide-stream-force step,
blowing-agent injection, pressure-Laplacian rupture criterion and gas
labelling, behind the C ABI of include/lbm.h.

``lbm`` is the thin ctypes binding; import it explicitly (it needs the built
CUDA library)."""
__all__ = ["lbm", "workloads"]
