"""GB300-native evaluation of parton distribution functions and alpha_s.

The hot path of PDFFlow (arXiv:2009.06635): batched x f(x, Q^2) by
log-bicubic interpolation on (ln x, ln Q^2) grids with Q subgrids split at
flavour thresholds, continuation outside the grid, and log-cubic
alpha_s(Q^2).  The evaluation runs in hand-written sm_103a CUDA kernels
behind the C ABI of include/pdf_gb300.h; this package is its Python binding.

    from paper_2009_06635_gb300 import pdf_load_grid, xfxq2_all_flavours, synthetic
"""
from . import synthetic
from ._native import PdfError
from .pdf import (Grid, XfxQ2AllFlavours, alphas_q, alphas_q2, pdf_grid_set_values, pdf_load_grid, pdf_mc_event,
                  xfxq2, xfxq2_all_flavours, xfxq2_all_flavours_diff, xfxq2_all_flavours_host,
                  xfxq2_all_flavours_vjp, xfxq2_all_members, xfxq2_all_flavours_alphas,
                  McResult, pdf_mc_integrate, pdf_load_lhapdf, read_lhapdf, scratch_limit,
                  set_scratch_limit)

__all__ = ["synthetic", "PdfError", "Grid", "pdf_load_grid", "xfxq2", "xfxq2_all_flavours",
           "alphas_q", "alphas_q2", "pdf_mc_event", "xfxq2_all_flavours_host", "xfxq2_all_flavours_vjp",
           "pdf_grid_set_values", "XfxQ2AllFlavours", "xfxq2_all_flavours_diff", "xfxq2_all_members",
           "xfxq2_all_flavours_alphas", "McResult", "pdf_mc_integrate",
           "pdf_load_lhapdf", "read_lhapdf", "set_scratch_limit", "scratch_limit"]
