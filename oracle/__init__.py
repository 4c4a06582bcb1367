"""FP64 CPU oracle for the multi-phenotype genome scan of TorchGWAS (arXiv 2604.21095).

TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the bench's CPU baseline
call it; the library and its Python binding never import it, and it imports
nothing from them. It is plain NumPy in float64, slow and direct:

* decode.py  - PLINK 1 .bed 2-bit calls and 8-bit dosages, exact integer marker
               statistics and mean imputation.
* panel.py   - the covariate basis Q (Householder QR of [1, C] with rank detection),
               the residualised panel of Eq. 1 and its unit-norm standardisation (Section 2.2).
* ols.py     - per-marker OLS of every phenotype on [1, C, g] solved directly, the
               projected form (Eq. 2 and Eq. 3 after projecting g on Q as well), and the
               paper's printed form (g only standardised, df = N - 2).
* pvalue.py  - two-sided Student-t p-values through the regularised incomplete beta
               function, evaluated in log space (Section 2.2: t converted to P values).
* scan.py    - the whole scan: statistics for every (marker, phenotype), hits above a
               -log10 p threshold and the best marker per phenotype; a panel may be
               prepared on the subset of samples its phenotypes are observed on.

Every function is pinned by tests under tests/ against closed forms, brute force on
tiny inputs, invariants or published table values; none is marked "parity unpinned".
"""
from .decode import decode_2bit, decode_u8, impute, marker_stats  # noqa: F401
from .panel import design_matrix, householder_basis, residualise  # noqa: F401
from .ols import ols_direct, ols_paper, ols_projected  # noqa: F401
from .pvalue import log_betainc, mlog10p_from_r, mlog10p_from_t  # noqa: F401
from .scan import best_per_phenotype, hits, prepare_panel, scan  # noqa: F401
