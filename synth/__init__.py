"""Seeded synthetic inputs for HHL state-vector simulation.

This module only *makes inputs*: power-grid matrices and right-hand sides, Haar-random gate
matrices with random target qubits, and random initial state vectors.  It holds none of the
simulation method's arithmetic (no gate application, no HHL circuit construction, no readout),
so that both the FP64 CPU oracle and the CUDA library can consume the same inputs without
sharing any code of the method.

The paper's workloads are IEEE 14/30-bus power-flow systems taken from MATPOWER (Sec. IV),
which are not available here; the reduced DC susceptance matrices below stand in for them:
a connected random graph, line susceptances uniform in [5, 20] p.u., weighted Laplacian with
the slack bus (bus 0) removed, which is symmetric positive definite.
"""
from .grids import (  # noqa: F401
    random_connected_graph,
    reduced_laplacian,
    grid_system,
    contingency_system,
    spectral_snap,
    random_rhs,
)
from .gates import haar_unitary, random_targets, gate_microbench_list  # noqa: F401
from .states import (  # noqa: F401
    counter_uniform_np,
    gaussian_state_np,
    gaussian_state_torch,
    gaussian_amplitudes_at,
    STATE_SCALE_NOTE,
)
from .acgrid import ac_case  # noqa: F401
from .workloads import (  # noqa: F401
    hhl7_problem,
    hhl27_problem,
    batched_problems,
    serving_stream,
)
