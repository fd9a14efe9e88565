// The comparators of Sec. 5 on the GPU: the preconditioner pass sequences for the circulant TBAN
// preconditioner F_C ("C-GMRES", length-n DFTs by Bluestein in place of the sine transforms) and for
// no preconditioner ("GMRES"), instantiated here so they compile beside the main solver.
#include "precon.cuh"

namespace rfnse {

RFNSE_PRECON_VARIANTS(RFNSE_PRECON_SIG, 1)
RFNSE_PRECON_VARIANTS(RFNSE_PRECON_SIG, 2)

}  // namespace rfnse
