"""Error type shared by the oracle modules (test infrastructure only)."""


class OracleError(Exception):
    """Raised with a status name matching the C ABI's ``pgcp_status`` codes.

    ``code`` is one of: ARG, NONMANIFOLD, TOPOLOGY, SCHEDULE, DEGENERATE,
    NUMERIC.
    """

    def __init__(self, code: str, msg: str):
        super().__init__(f"{code}: {msg}")
        self.code = code
