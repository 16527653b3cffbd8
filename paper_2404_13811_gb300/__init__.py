"""GB300 (sm_103a) implementation of the Multiscale Robin Coupled Method with
Oversampling and Smoothing (arXiv 2404.13811): C-ABI library ``libmrcm.so``
and its thin Python binding.  The CUDA library is loaded on first use and a
missing build raises instead of falling back to anything else."""

__all__ = ["inputs"]
