"""CPU FP64 oracle for RAS/ORAS-preconditioned FGMRES on the closest point method (CPM).

TEST INFRASTRUCTURE, NOT PRODUCT CODE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run anything in
this package. It shares no code with the CUDA path (``paper_1909_08734_gb300``) and imports
nothing from it; the only module both sides use is ``workloads`` (seeded inputs).

Source: May, Haynes & Ruuth, "Schwarz solvers and preconditioners for the closest point
method" (arXiv:1909.08734). Every function cites the section / equation it follows.
Plain NumPy/SciPy in FP64, written for readability, not speed.

Modules
  geometry   closest-point functions and normals (Sec. 2.1, CP definition)
  band       tube-radius active set, ghost set, canonical order (Sec. 2.1)
  interp     barycentric Lagrange extension matrix E (Sec. 2.1, Fig. 1)
  operator   stabilised CPM matrix A = cI - Lap_S^h (Eq. impLapBel)
  partition  coordinate bisection, overlap growth, node sets, cross points (Secs. 3-4, 5.2.2)
  local      RAS / ORAS local operators (Eqs. simpleRAS, localOP, naConorm, robfo)
  schwarz    restricted additive Schwarz preconditioner / solver (Eq. algRAS)
  krylov     right-preconditioned flexible GMRES(m) with CGS2 (Sec. 2.2)
  problems   one-call setup of a named workload

Parity status (what pins each part lives in tests/test_oracle_*.py):
  band, interp, operator, partition, RAS, FGMRES: pinned.
  ORAS local operator: pinned in its parts (argmin, conormal identity, cross points,
  Robin scaling), by the one-subdomain / converged-solution properties, and as a whole
  (tests/test_oracle_robin.py): with exact Robin data on a spherical cap the local solution
  converges at first order under readings R1 and R3 (Table 1's order), d.q uses the normal at
  CP_{S_j}, alpha -> infinity gives the Dirichlet transmission of Sec. 5.1, the two readings
  differ in the boundary rows only, and a planted wrong Robin weight fails.  On a triangulated
  surface (face normals) the Robin rows stay pinned only by the solution properties.
"""
