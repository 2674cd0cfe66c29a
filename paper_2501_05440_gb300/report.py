"""Reporting helpers for benchmark lines (no transport arithmetic here)."""


def core_equivalency(cpu_cores, cpu_runtime, n_gpus, gpu_runtime):
    """Effective CPU cores per GPU, Eq. 1: (#CPU cores x CPU run time) / (#GPUs x GPU run time).

    With throughputs instead of run times for the same work, pass the inverse
    rates (run time is proportional to 1/throughput)."""
    return (cpu_cores * cpu_runtime) / (n_gpus * gpu_runtime)
