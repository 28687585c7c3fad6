"""GB300 Cholesky / Cholesky-adjoint / GP-likelihood library (binding placeholder)."""
