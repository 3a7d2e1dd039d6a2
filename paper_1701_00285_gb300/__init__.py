"""GB300 multilevel BLUP (arXiv:1701.00285): C-ABI library libmlblup.so and
its Python binding.  See include/mlblup.h for the boundary."""
from .binding import Context, MLBError, covariance, lib  # noqa: F401
