"""GB300 (sm_103a) sparse fusion: a GPU inspector and a fused persistent executor for
SpTRSV->SpMV, SpIC0->SpTRSV and SpMV->SpTRSV, behind the C ABI of include/sparsefusion.h.

The CUDA library is loaded lazily by ``paper_2111_12238_gb300.sparsefusion``; importing the
package itself loads nothing, so the seeded input generators (``inputs``) are usable
without a GPU.
"""
__all__ = ["inputs", "sparsefusion"]
