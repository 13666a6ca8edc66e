"""FP64 CPU oracle (test infrastructure only): see ``oracle.t_energy``."""
