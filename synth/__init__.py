"""Seeded synthetic galaxy / random catalogs shared by the tests, the oracle
legs and the benchmark.  This package holds only input generation (random
draws, geometry, the lognormal field used to place galaxies); none of the
estimators' arithmetic lives here."""
from .catalogs import (Catalog, uniform_cube_catalog, lognormal_cap_catalog,  # noqa: F401
                       snapped_catalog)
